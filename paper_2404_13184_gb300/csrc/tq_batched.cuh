// Batched tensor-core passes (the FP64-accurate pass of tq_apply_oz.cu and
// the split pass of tq_apply_tc.cu): the job tables a launch takes, shared by
// the kernels and the batch engine that builds them.
#pragma once

#include "tq_device.cuh"

namespace tq {

// One (state, fused block) of a batched pass. The units of all jobs of a
// launch are numbered one after another; unit0 is this job's first.
struct OzJob {
  double2* rho;              // the state's vec(rho), Hermitian mode
  const double2* S;          // the block's fused FP64 superoperator
  ApplyParams p;             // width 2 (a width-1 block: q[1] is the embedding qubit)
  int embed;                 // 1: S is 4 x 4, applied as S (x) I
  int pad_;
  unsigned long long unit0;  // first unit of this job in the launch
};

// Work units (half tiles of 16 x 16 canonical groups) of one pass on n qubits.
unsigned long long oz_units(int n);

// The job entry of block (S, p) of the state at rho, unit0 left 0; false when
// the block is not eligible for the pass.
bool oz_job(double2* rho, const double2* S, const ApplyParams& p, OzJob* out);

// One batched pass over jobs[0 .. n_jobs) (device table, n_units in total).
cudaError_t launch_batch_oz(const OzJob* jobs, int n_jobs, unsigned long long n_units, int num_sms,
                            cudaStream_t st);

// The same for the split pass (complex64 states, FP32 superoperators).
struct TcJob {
  float2* rho;               // the state's vec(rho), Hermitian mode
  const float2* S;           // the block's fused superoperator (FP32)
  ApplyParams p;             // width 2 (a width-1 block: q[1] is the embedding qubit)
  int embed;                 // 1: S is 4 x 4, applied as S (x) I
  int pad_;
  unsigned long long unit0;  // first unit of this job in the launch
};

// Units of one split pass on n qubits (the same half tiles).
unsigned long long tc_units(int n);

bool tc_job(float2* rho, const float2* S, const ApplyParams& p, TcJob* out);

cudaError_t launch_batch_tc(const TcJob* jobs, int n_jobs, unsigned long long n_units, int num_sms,
                            cudaStream_t st);

}  // namespace tq
