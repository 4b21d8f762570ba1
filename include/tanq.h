/*
 * tanq.h -- C ABI of a GB300 (sm_103a) noisy density-matrix simulator.
 *
 * The library computes, on one GPU, the problem of TANQ-Sim (arXiv
 * 2404.13184) Sec. 2.1, Eq. 2: given an n-qubit density matrix rho_in and a
 * sequence of gates and noise channels G_0 .. G_{m-1},
 *     rho_out = G_{m-1}( ... G_1(G_0 rho_in G_0^dag) G_1^dag ... ) G_{m-1}^dag,
 * where a noisy G is a Kraus set {K_i} acting as rho -> sum_i K_i rho K_i^dag
 * (Sec. 3.1, Kraus sum).
 *
 * Method (Sec. 3.1, Eq. "sp"): rho is stored as vec(rho), the column-stacked
 * 4^n vector (vec index v = r + c * 2^n for rho[r][c]); every op becomes the
 * superoperator S = sum_i conj(K_i) (x) K_i; consecutive ops are fused into
 * dense superoperators on at most 4 qubits (Sec. 3.3, generalised); each
 * fused block is applied to all 4^n entries by gathering the 4^k entries of
 * every group at the target bit positions (q_j and q_j + n), multiplying by
 * the 4^k x 4^k superoperator and scattering back (Sec. 3.1, C1/C2 update,
 * generalised from k = 1, 2 to k <= 4).
 *
 * Conventions used by every entry point:
 *  - qubit q is bit q of the row index r and of the column index c, so it is
 *    bits q and q + n of the vec index;
 *  - a k-qubit matrix acts on an ordered list qubits[0..k-1]; bit j of its
 *    local row/column index is qubit qubits[j] (qubits[0] is the least
 *    significant local bit);
 *  - matrices are 2^k x 2^k complex, row-major, interleaved (re, im) doubles:
 *    element (i, j) is at [2*(i*2^k + j)] (re) and [2*(i*2^k + j) + 1] (im);
 *  - readouts are reduced in FP64 in a fixed order (deterministic for a given
 *    n and precision).
 *
 * Ownership: every input array is owned by the caller and copied (or fully
 * consumed) before the call returns; output arrays are caller-allocated. A
 * tq_state owns its device buffers until tq_free (except for the rho buffer
 * passed to tq_create_on, which stays the caller's).
 *
 * Streams: apply calls enqueue work on the state's CUDA stream and return
 * without waiting; readouts (tq_trace, tq_expect_z, tq_probs, tq_get_rho)
 * wait for the stream before returning.
 *
 * Errors: every call returns a tq_status. Argument errors leave the state
 * unchanged. After a CUDA error the state is poisoned and every later call
 * on it returns TQ_ERR_STATE; only tq_free is then valid.
 */
#ifndef TANQ_H
#define TANQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tq_state tq_state; /* opaque; owns the device copy of vec(rho) */

typedef enum {
  TQ_FP64 = 0,  /* rho complex128, superoperator products in FP64 */
  TQ_SPLIT = 1  /* rho complex64, products in FP32 (FP64 superoperator build,
                   fusion, trace renormalisation and readouts). Width-2
                   blocks on a Hermitian state run on the tcgen05 tensor
                   cores: each FP32 operand split into three BF16 terms,
                   six term products accumulated in FP32 (Sec. 3.2 maps the
                   update onto tensor cores) */
} tq_precision;

typedef enum {
  TQ_OK = 0,
  TQ_ERR_ARG = 1,         /* bad size, null pointer, unknown kind/name, bad parameter */
  TQ_ERR_QUBIT = 2,       /* qubit index out of range or repeated */
  TQ_ERR_OOM = 3,         /* device or pinned host allocation failed */
  TQ_ERR_CUDA = 4,        /* a CUDA call failed; the state is now poisoned */
  TQ_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  TQ_ERR_STATE = 6,       /* the state was poisoned by an earlier CUDA error */
  TQ_ERR_UNSUPPORTED = 7  /* valid request this build does not provide */
} tq_status;

/* Named gates (textbook definitions; Sec. 4 Table 2 lists the gate family).
 * Parameters: RX/RY/RZ/RZZ take params[0] = angle theta with
 * RX = exp(-i theta X/2), RY = exp(-i theta Y/2), RZ = diag(e^{-i theta/2},
 * e^{i theta/2}), RZZ = exp(-i theta Z(x)Z/2). SU2 takes params[0..3] = four
 * real numbers (not all zero) normalised to a unit quaternion (a, b, c, d):
 * U = [[a+ib, c+id], [-c+id, a-ib]]; four i.i.d. normal draws give a
 * Haar-random SU(2). CX/CZ: qubits[0] is the control, qubits[1] the target. */
typedef enum {
  TQ_GATE_ID = 0, TQ_GATE_H, TQ_GATE_X, TQ_GATE_Y, TQ_GATE_Z, TQ_GATE_S,
  TQ_GATE_SDG, TQ_GATE_T, TQ_GATE_TDG, TQ_GATE_SX, TQ_GATE_RX, TQ_GATE_RY,
  TQ_GATE_RZ, TQ_GATE_SU2,
  TQ_GATE_CX = 32, TQ_GATE_CZ, TQ_GATE_SWAP, TQ_GATE_RZZ
} tq_gate;

/* Named noise channels (Sec. 3.5). k is the number of qubits the op lists.
 *  DEPOLARIZING  params[0] = p in [0, 4^k/(4^k-1)]: rho -> (1-p) rho +
 *                p (I/2^k) (x) Tr_Q(rho), given as the 4^k Pauli Kraus
 *                operators sqrt(1 - p (4^k-1)/4^k) I and sqrt(p/4^k) P;
 *                k in 1..2.
 *  AMPLITUDE_DAMPING params[0] = gamma in [0,1]: K0 = [[1,0],[0,sqrt(1-g)]],
 *                K1 = [[0,sqrt(g)],[0,0]]; k = 1.
 *  PHASE_DAMPING params[0] = lambda in [0,1]: K0 = [[1,0],[0,sqrt(1-l)]],
 *                K1 = [[0,0],[0,sqrt(l)]]; k = 1.
 *  THERMAL       params = (t, T1, T2), t >= 0, T1 > 0, 0 < T2 <= 2 T1:
 *                zero-temperature relaxation rho00 += (1-e^{-t/T1}) rho11,
 *                rho11 *= e^{-t/T1}, rho01 *= e^{-t/T2}; applied
 *                independently to each of the k (1..2) listed qubits.
 *  RESET         no parameters: the qubit is reset to |0>, K0 = |0><0|,
 *                K1 = |0><1|; k = 1 (the reset gate announced in Sec. 3,
 *                whose section the paper does not contain). */
typedef enum {
  TQ_CH_DEPOLARIZING = 0,
  TQ_CH_AMPLITUDE_DAMPING = 1,
  TQ_CH_PHASE_DAMPING = 2,
  TQ_CH_THERMAL = 3,
  TQ_CH_RESET = 4
} tq_channel;

typedef enum {
  TQ_OP_UNITARY = 0,  /* mats = one 2^k x 2^k matrix U: rho -> U rho U^dag (Eq. 1) */
  TQ_OP_KRAUS = 1,    /* mats = m matrices K_i: rho -> sum_i K_i rho K_i^dag; K need
                         not be trace preserving (Sec. 2.1: G need not be unitary) */
  TQ_OP_GATE = 2,     /* name = tq_gate, params as documented there */
  TQ_OP_CHANNEL = 3   /* name = tq_channel, params as documented there */
} tq_op_kind;

/* One circuit op. For UNITARY/KRAUS, mats points to m (1 for UNITARY)
 * matrices in the layout above; for GATE/CHANNEL it is ignored. */
typedef struct tq_op {
  int32_t kind;        /* tq_op_kind */
  int32_t k;           /* number of qubits, 1..4 */
  int32_t qubits[4];   /* qubits[0..k-1], distinct, each in [0, n) */
  int32_t m;           /* number of Kraus matrices (KRAUS), else ignored */
  int32_t name;        /* tq_gate (GATE) or tq_channel (CHANNEL) */
  double params[4];
  const double* mats;
} tq_op;

/* ---- states ----------------------------------------------------------- */

/* Create rho = |0..0><0..0| for n qubits (1 <= n <= 16; device memory
 * 16 * 4^n bytes in TQ_FP64, 8 * 4^n in TQ_SPLIT), working on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream) of the current device. */
tq_status tq_create(int n_qubits, int precision, void* cuda_stream, tq_state** out);

/* As tq_create, but vec(rho) lives in caller-owned device memory `rho_dev`
 * of `bytes` bytes (>= 16*4^n FP64 / 8*4^n SPLIT, 256-byte aligned), for
 * example a tensor from PyTorch's caching allocator. The buffer is
 * initialised to |0..0><0..0| and must outlive the state. */
tq_status tq_create_on(int n_qubits, int precision, void* cuda_stream, void* rho_dev,
                       size_t bytes, tq_state** out);

void tq_free(tq_state* s);

/* Number of qubits and precision of a state (TQ_ERR_ARG on NULL). */
tq_status tq_info(const tq_state* s, int* n_qubits, int* precision);

/* Reset rho to |0..0><0..0| (asynchronous). */
tq_status tq_reset(tq_state* s);

/* Device address of vec(rho) (complex128 or complex64, interleaved), for
 * zero-copy interop on the state's stream. All 4^n entries are current once
 * work enqueued before this call completes (in Hermitian mode the lower
 * triangle is filled first, asynchronously on the stream). */
tq_status tq_rho_device_ptr(tq_state* s, void** out);

/* Hermitian mode (FP64 states; on by default). Every op is a Kraus map,
 * which keeps rho = rho^dagger, so the group with row-rest bits a and
 * column-rest bits b is the conjugate transpose of group (b, a): only the
 * groups with a <= b are computed and only entries with row <= column are
 * kept current, halving the work of every apply pass. The diagonal, hence
 * every readout, is always current; tq_get_rho and tq_rho_device_ptr fill
 * the lower triangle first. The mode is active only while rho is known to
 * be Hermitian: from tq_create/tq_reset on, and after tq_set_rho only if
 * max |rho - rho^dagger| <= 4 eps max |rho| (checked on the GPU). on = 0
 * turns it off (full updates). */
tq_status tq_set_hermitian(tq_state* s, int on);

/* *active = 1 if apply passes currently use Hermitian mode. */
tq_status tq_is_hermitian_mode(const tq_state* s, int* active);

/* Products of the FP64 apply passes (TQ_FP64 states).
 *  TQ_ENGINE_DFMA    FP64 fused multiply-adds on the CUDA cores (dense
 *                    kernels, or row lists of the nonzero superoperator
 *                    entries for structured blocks).
 *  TQ_ENGINE_TENSOR  blocks of width <= 2 in Hermitian mode on registers of
 *                    n >= 6 qubits run on the tcgen05 tensor cores: every
 *                    operand (the group's 32 real values, each real row of
 *                    the superoperator) is cut into seven balanced 8-bit
 *                    digits of a 54-bit fixed-point number aligned to the
 *                    largest exponent of its group or row; the digit
 *                    products, on the tensor cores with FP16 operands, are
 *                    summed EXACTLY in FP32 per digit order (Ozaki-style
 *                    error-free splitting) for orders 0..7 (orders >= 8,
 *                    ~2^-53 of order 0, dropped), and recombined in 64-bit
 *                    integers, so each output carries the operands' rounding
 *                    at 2^-55 of their alignment, ~2^-53 from the dropped
 *                    orders and one final rounding: FP64 accuracy relative
 *                    to the largest entry of its group (the paper's FP64
 *                    tensor-core C2 update, Sec. 3.2, mapped onto the
 *                    tensor cores this GPU
 *                    has). A width-1 block runs as S (x) I on two qubits.
 *                    Other blocks use the DFMA kernels.
 *  TQ_ENGINE_AUTO    the library's choice (the default): the tensor cores
 *                    wherever TQ_ENGINE_TENSOR applies (measured on GB300:
 *                    7.4 ms per 15-qubit width-2 pass against 18.1 ms for
 *                    the DFMA row-list kernel).
 * The engine is read when passes are enqueued (a device program's captured
 * graph is recaptured when it changes). */
typedef enum { TQ_ENGINE_AUTO = 0, TQ_ENGINE_DFMA = 1, TQ_ENGINE_TENSOR = 2 } tq_fp64_engine;
tq_status tq_set_fp64_engine(tq_state* s, int engine);

/* *on_tensor = 1 if the state's FP64 passes of widths <= 2 run on the tensor
 * cores (TQ_ENGINE_TENSOR, or TQ_ENGINE_AUTO where the library chooses them). */
tq_status tq_fp64_on_tensor(const tq_state* s, int* on_tensor);

/* Copy vec(rho) out to / in from host memory: 2 * 4^n doubles, interleaved
 * (re, im) in vec order (index r + c 2^n). Split states convert from/to
 * complex64. tq_get_rho waits for the stream. */
tq_status tq_get_rho(tq_state* s, double* out);
tq_status tq_set_rho(tq_state* s, const double* in);

/* ---- evolution -------------------------------------------------------- */

/* rho -> U rho U^dag with U a 2^k x 2^k matrix on qubits[0..k-1], 1 <= k <= 4
 * (Eq. 1; applied as vec(rho) -> (conj(U) (x) U) vec(rho), Sec. 3.1). */
tq_status tq_apply_gate(tq_state* s, const int* qubits, int k, const double* U);

/* rho -> sum_{i<m} K_i rho K_i^dag, K_i 2^k x 2^k on qubits[0..k-1]
 * (Sec. 3.1 Kraus sum; superoperator S = sum_i conj(K_i) (x) K_i). */
tq_status tq_apply_kraus(tq_state* s, const int* qubits, int k, int m, const double* K);

/* Run ops[0..n_ops-1] in order (Eq. 2). Ops are fused into blocks of at most
 * max_fuse_width qubits (1..4) by merging each op into the latest block that
 * shares a qubit with it when the union stays within the width and no
 * later block touches those qubits (Sec. 3.3, generalised); 0 applies every
 * op as its own pass (no fusion); -1 lets the library's cost model choose
 * the width for this n and precision. Superoperators are built and fused in
 * FP64 on the GPU. Asynchronous. If n_blocks_out is not NULL it receives the
 * number of fused blocks applied. */
tq_status tq_run_circuit(tq_state* s, const tq_op* ops, size_t n_ops, int max_fuse_width,
                         size_t* n_blocks_out);

/* Failure-detection hook for tests (the paper has no counterpart): the
 * MMA-completion waits of the tensor-core passes (width-2 blocks of a
 * TQ_SPLIT state in Hermitian mode, and the FP64 passes of
 * TQ_ENGINE_TENSOR) give up after max_tries try-wait rounds
 * (0 restores the default, ~seconds); with skip_mma != 0 the passes
 * launched afterwards issue neither their MMAs nor the commit, so their
 * first wait runs out with nothing in flight and the next synchronising
 * readout of that state returns TQ_ERR_TIMEOUT (the state is poisoned)
 * while the CUDA context stays usable. Process-wide; read at each launch
 * (a device program's captured graph keeps the values it was captured
 * with). TQ_ERR_ARG if max_tries < 0. */
tq_status tq_test_tc_wait_limit(long long max_tries, int skip_mma);

/* ---- readouts (FP64 reductions over the diagonal, Sec. 2.1) ------------ */
/* The synchronising readouts (tq_trace, tq_expect_z, tq_probs,
 * tq_probs_readout, tq_sample, tq_measure, tq_get_rho) of a TQ_SPLIT state
 * that has run a tensor-core pass also report TQ_ERR_TIMEOUT, and poison the
 * state, if a bounded wait for that pass's MMAs ran out (a pass that did not
 * complete; its results are not valid). */

/* Tr(rho) = sum_x rho[x][x]. */
tq_status tq_trace(tq_state* s, double* re, double* im);

/* out[i] = Re Tr(rho Z_{masks[i]}) for i < n_masks (Z on every qubit whose
 * bit is set in the mask; mask 0 gives Re Tr rho). In TQ_SPLIT the values
 * are divided by Re Tr(rho) (trace renormalisation). */
tq_status tq_expect_z(tq_state* s, const uint64_t* masks, int n_masks, double* out);

/* out[x] = Re rho[x][x] for x < 2^n: the probabilities of measuring every
 * qubit in the computational basis (renormalised to sum 1 in TQ_SPLIT). */
tq_status tq_probs(tq_state* s, double* out);

/* ---- compiled programs (ops resident in device memory) ------------------ */

typedef struct tq_program tq_program; /* opaque; owns device copies of its tables */

/* Validate ops for an n-qubit register of the given precision, plan the
 * fusion (max_fuse_width as in tq_run_circuit; the automatic width follows
 * the cost model of the default FP64 engine, TQ_ENGINE_AUTO, whereas
 * tq_run_circuit follows the state's engine) and upload the Kraus sets and
 * plan tables to device memory once (synchronously). Running the program
 * then re-does the superoperator build, the fusion and the apply passes from
 * device-resident inputs with no host copies. */
tq_status tq_program_create(int n_qubits, int precision, const tq_op* ops, size_t n_ops,
                            int max_fuse_width, tq_program** out);

/* Enqueue the program on the state's stream (asynchronous). The state must
 * have the program's n and precision (TQ_ERR_ARG otherwise). One program
 * may be run on several states, but not concurrently on two streams nor
 * from two host threads at once.
 *
 * The whole launch sequence is captured once into a CUDA graph and
 * replayed. The graph bakes in the state's density-matrix buffer and
 * whether Hermitian mode applies on entry. A run with another buffer or
 * other entry flags recaptures it; the first run after a change pays the
 * capture. With profiling on (tq_profile_enable) the launches are made
 * one by one instead. For registers of at most 8 qubits whose blocks are
 * at most 2 qubits wide, the apply passes are one kernel on a
 * thread-block cluster holding rho in distributed shared memory, with a
 * cluster barrier between blocks (Sec. 3.1 apply step). */
tq_status tq_program_run(tq_state* s, const tq_program* p);

/* Number of ops, of fused blocks, widest block, and the bytes of its device
 * tables (Kraus sets and plan: what tq_run_circuit copies host-to-device
 * for the same ops). Any output pointer may be NULL. */
tq_status tq_program_info(const tq_program* p, size_t* n_ops, size_t* n_blocks, int* max_width,
                          size_t* table_bytes);

void tq_program_free(tq_program* p);

/* Device-side readout: out_dev[i] = Re Tr(rho Z_{masks_dev[i]}) (divided by
 * Re Tr rho in TQ_SPLIT) for i < n_masks <= 16; masks_dev and out_dev are
 * device pointers. Asynchronous on the state's stream. */
tq_status tq_expect_z_device(tq_state* s, const uint64_t* masks_dev, int n_masks, double* out_dev);

/* ---- batched execution (many independent circuits, one persistent launch) --
 * Jobs are independent circuits, each on its own |0..0><0..0| state of n
 * qubits (1..16) of the batch's precision. tq_batch_run resets every state,
 * builds and fuses all superoperators (two launches over all jobs), applies
 * every job's fused blocks in ONE persistent kernel launch, and reduces each
 * job's trace and <Z_mask> values; the sequence is captured as a CUDA graph
 * on the first run (on a private stream) and replayed by later runs on the
 * batch's stream. Small registers (vec(rho) <= 64 KiB) run their whole
 * circuit in shared memory; larger ones are split into tiles whose order
 * respects each job's block sequence (single-kernel execution, Sec. 3.4 and
 * Listing 2, applied across independent circuits). */

typedef struct tq_batch tq_batch;

/* An empty batch working on `cuda_stream` (NULL: legacy default stream). */
tq_status tq_batch_create(int precision, void* cuda_stream, tq_batch** out);

/* Add a job: ops as in tq_run_circuit, fused with max_fuse_width in
 * {-1, 0, 1, 2} (-1: cost model, capped at 2; 3 and 4 give
 * TQ_ERR_UNSUPPORTED, as does any op on more than 2 qubits); masks: up to 16
 * Z-masks to read out after the run. *job_out receives the job index. */
tq_status tq_batch_add(tq_batch* b, int n_qubits, const tq_op* ops, size_t n_ops, int max_fuse_width,
                       const uint64_t* masks, int n_masks, int* job_out);

/* Entries per tile (2^tile_log2) for the jobs of n_qubits qubits: the work
 * granularity of the persistent kernel, normally set by the autotuner. */
tq_status tq_batch_set_tile(tq_batch* b, int n_qubits, int tile_log2);

/* Engine of the batch's tile jobs (vec(rho) > 64 KiB; tq_fp64_engine,
 * default TQ_ENGINE_AUTO). On the batched tensor-core pass of its precision
 * a tile job whose blocks are all of width <= 2 runs instead of on the
 * persistent kernel: one launch per fusion round, each applying that
 * round's block of every such job (FP64: the FP64-accurate digit pass
 * tq_set_fp64_engine describes; split: the three-term BF16 pass of single
 * split states; width-1 blocks as S (x) I). FP64 takes it with
 * TQ_ENGINE_AUTO or TQ_ENGINE_TENSOR, split only with TQ_ENGINE_TENSOR (the
 * faster choice measured on GB300 in each precision; the split pass is the
 * more accurate one). Otherwise the persistent kernel runs every job (FP64
 * DFMA row lists; split FP32 Pauli-basis products on the CUDA cores).
 * Resident jobs always run on the persistent kernel. Takes effect at the
 * next run. */
tq_status tq_batch_set_fp64_engine(tq_batch* b, int engine);

/* Jobs of the last planned run on a batched tensor-core pass. */
tq_status tq_batch_tensor_jobs(const tq_batch* b, size_t* n_jobs);

/* Enqueue one run of every job (asynchronous). */
tq_status tq_batch_run(tq_batch* b);

/* Failure-detection hook for tests: every device-side wait of the batch
 * kernel gives up after max_spin polls (default 2e7, seconds), sets an error
 * flag and lets the kernel finish; with never_ready_job >= 0 that job's waits
 * can never be satisfied (the job stays on the persistent kernel), so a run
 * ends with TQ_ERR_TIMEOUT from tq_batch_wait while the CUDA context stays
 * usable. -1 restores normal waits. The tensor-core pass's waits follow
 * tq_test_tc_wait_limit and report through tq_batch_wait too. */
tq_status tq_batch_test_wait_limit(tq_batch* b, long long max_spin, int never_ready_job);

/* Wait for the last run; TQ_ERR_TIMEOUT if a bounded device-side wait ran
 * out (the results are then invalid). */
tq_status tq_batch_wait(tq_batch* b);

/* out[0..1] = Re, Im Tr(rho_job); out[2+i] = Re Tr(rho_job Z_{mask_i}) (divided
 * by Re Tr rho_job in TQ_SPLIT). Waits for the run. */
tq_status tq_batch_result(tq_batch* b, int job, double* out);

/* vec(rho_job) as 2*4^n interleaved doubles (waits for the run). */
tq_status tq_batch_get_rho(tq_batch* b, int job, double* out);

/* Jobs, work items of the persistent launch (tensor-core jobs not
 * included), bytes of all density matrices. */
tq_status tq_batch_info(const tq_batch* b, size_t* n_jobs, size_t* n_items, size_t* rho_bytes);

/* Algorithmic work of one run, counted on the device from the fused
 * superoperators of the last run (Sec. 3.1: one gather, product and scatter
 * per group). flops: per group of every block (canonical groups in
 * Hermitian mode), 8 real flops per complex multiply-add the apply kernel
 * issues -- FP64 counts nonzero superoperator entries only (its row lists
 * skip the zeros), split counts all -- except for width-2 blocks of tile
 * jobs that the kernel runs in the Pauli basis (real R' = T S T^dagger /
 * 16): FP64 row lists of R' count 4 flops per nonzero plus the 128 adds of
 * the basis changes, split (always in the Pauli basis, R' dense) 4 x 256 +
 * 128; blocks of jobs on a batched tensor-core pass count the dense
 * product (8 per entry of S). bytes: what the apply passes must move through
 * HBM: per block of a tile job one read and one write of the stored entries
 * (the upper triangle in Hermitian mode), per resident job one load and one
 * store of vec(rho). TQ_ERR_STATE before the first run; waits for the run. */
tq_status tq_batch_work(tq_batch* b, double* flops, double* bytes);

void tq_batch_free(tq_batch* b);

/* Autotuner of the batch engine: times every (fusion width in {1, 2},
 * entries per tile) candidate for n_qubits (2..14) at this precision on a
 * synthetic batch of random depolarised {H, RZ, RX, CX} circuits (depth
 * 64; about 2^24 density-matrix entries in total, and at least enough jobs
 * for ~8 work items per SM at the largest tile, at most 256) and returns
 * the fastest
 * (*ms_out: its time per run). With cache_path not NULL, a cached result for
 * this GPU name, precision and n is returned without timing, and a new
 * result is appended to the file ("<gpu> <precision> <n> <tile_log2>
 * <width> <ms>" per line). */
tq_status tq_autotune(int precision, int n_qubits, const char* cache_path, int* tile_log2_out,
                      int* width_out, double* ms_out);

/* The same for a batch that runs on the given engine (tq_fp64_engine, as
 * tq_batch_set_fp64_engine): the candidates run on that engine; results are
 * cached under "fp64" (tensor-core pass), "fp64-dfma", "split" (persistent
 * kernel) or "split-tc" (tq_autotune is this call with TQ_ENGINE_AUTO). */
tq_status tq_autotune_engine(int precision, int fp64_engine, int n_qubits, const char* cache_path,
                             int* tile_log2_out, int* width_out, double* ms_out);

/* ---- serving loop (continuous batching of circuit requests) --------------
 * Requests (independent circuits, each on its own |0..0><0..0|) wait in a
 * FIFO queue. A request is admitted, in order, when its density matrix fits
 * the rho budget (16*4^n bytes FP64, 8*4^n split; memory from a device arena
 * allocated once at creation) and a live slot is free; admission uploads its
 * tables and builds and fuses its superoperators (FP64, GPU). Each
 * tq_server_step is one tick: admit, then ONE persistent batch-kernel launch
 * that advances every live request by a quantum of fused blocks (about eight
 * 12-qubit passes' worth of entries, at least one block), then readouts of
 * the requests that finished, whose memory is returned. rho stays resident
 * between ticks; requests submitted while others run join the next tick. */

typedef struct tq_server tq_server;

/* rho_budget_bytes: device memory for the live density matrices;
 * table_budget_bytes: for their Kraus sets, plans and superoperators;
 * max_live: live requests at most. Allocates both budgets up front. */
tq_status tq_server_create(int precision, void* cuda_stream, size_t rho_budget_bytes,
                           size_t table_budget_bytes, int max_live, tq_server** out);

/* Queue a request (ops and masks as in tq_batch_add; widths <= 2).
 * TQ_ERR_OOM if its density matrix can never fit the budget. */
tq_status tq_server_submit(tq_server* s, int n_qubits, const tq_op* ops, size_t n_ops,
                           int max_fuse_width, const uint64_t* masks, int n_masks, int* request_id);

/* One tick (waits for it). Outputs (may be NULL): live requests, queued
 * requests, requests finished in this tick. */
tq_status tq_server_step(tq_server* s, int* n_live, int* n_queued, int* n_finished);

/* Pipelined tick: first collect the tick launched by the previous call
 * (waits for it; *n_finished = requests it finished, whose results
 * tq_server_poll now returns), then admit and launch the next tick and
 * return without waiting, so the caller's own work (building and
 * submitting requests, polling) overlaps the GPU. *n_live and *n_queued
 * describe the state after the launched tick. Bounded-wait timeouts of a
 * tick are reported by the call that collects it. Mixing with
 * tq_server_step is allowed: tq_server_step collects a pending tick first. */
tq_status tq_server_step_async(tq_server* s, int* n_live, int* n_queued, int* n_finished);

/* Products of FP64 requests (as tq_set_fp64_engine): with the tensor
 * cores, requests of at least 12 qubits advance through the single-state
 * tensor-core pass, one launch per fused block after the tick's batch
 * kernel (split requests of at least 12 qubits always do, their width-2
 * blocks on the split tensor-core pass); smaller requests stay in the
 * persistent batch kernel. Applies to ticks launched afterwards. */
tq_status tq_server_set_fp64_engine(tq_server* s, int engine);

/* GPU time of all collected ticks (CUDA events around each tick's
 * admission, apply and readout work), in milliseconds. */
tq_status tq_server_gpu_ms(const tq_server* s, double* ms);

/* *state: 0 queued, 1 live, 2 done; when done, out (if not NULL) receives
 * 2 + n_masks doubles as in tq_batch_result. */
tq_status tq_server_poll(tq_server* s, int request_id, int* state, double* out);

/* Bytes of live density matrices, ticks run, fused blocks applied. */
tq_status tq_server_info(const tq_server* s, size_t* rho_live_bytes, unsigned long long* ticks,
                         unsigned long long* blocks_applied);

void tq_server_free(tq_server* s);

/* ---- allocation-free readout ---------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not let the library allocate device memory: a host program whose
 * HBM is entirely owned by another allocator (such as PyTorch's caching
 * allocator in a serving process), or one that cannot afford the device-wide
 * synchronisation that cudaFree implies.
 *
 * Same result as tq_expect_z_device, but for a caller-owned vec(rho) (no
 * tq_state): out_dev[i] = Re Tr(rho Z_{masks_dev[i]}) for i < n_masks, divided
 * by Re Tr(rho) when precision is TQ_SPLIT. rho_dev holds 4^n_qubits complex
 * entries (complex128 for TQ_FP64, complex64 for TQ_SPLIT) in vec order;
 * masks_dev and out_dev are device arrays of n_masks entries. Enqueued on
 * cuda_stream; returns without waiting.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (at most 152 x 18 partial sums plus the totals, 22,144 bytes) is a fixed
 * device array inside the library, present on every GPU that loads the
 * library until the process exits. Limits: 1 <= n_masks <= 16 and
 * 1 <= n_qubits <= 16; larger requests return TQ_ERR_ARG. The first call on
 * each device looks up that array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of the process; make that first call before any
 * stream capture, and do not call this entry point again on a device after
 * cudaDeviceReset (a new context may place the array elsewhere, and the kept
 * address would then be stale). All calls share the one
 * array, so calls whose work overlaps on the GPU (different streams, or
 * different host threads without ordering) race and give wrong results;
 * order them on one stream. Nothing in the array needs clearing between
 * calls: each call writes every partial it later reads. */
tq_status tq_expect_z_noalloc(const void* rho_dev, int n_qubits, int precision,
                              const uint64_t* masks_dev, int n_masks, double* out_dev,
                              void* cuda_stream);

/* ---- pipe-rate probes (roofline denominators) ---------------------------
 * The paper has no counterpart; these measure the issue rates the apply
 * kernels' rooflines are taken against, where a copy benchmark or a cuBLAS
 * GEMM gives none: the FP64 FMA pipe (the FP64 apply passes are bound by
 * it), the FP64 tensor path (mma.sync m8n8k4, the paper's Sec. 3.2 mapping),
 * FP32 FMA, and two conversions to FP64. */
typedef enum {
  TQ_PIPE_DFMA = 0,        /* fma.rn.f64: 2 flops per FMA */
  TQ_PIPE_DMMA = 1,        /* mma.sync.m8n8k4.f64: 512 flops per warp instruction */
  TQ_PIPE_FFMA = 2,        /* fma.rn.f32: 2 flops per FMA */
  TQ_PIPE_CVT_F64_S64 = 3, /* cvt.rn.f64.s64: 1 op per conversion (each feeding the
                              next of its chain through one integer op) */
  TQ_PIPE_CVT_F64_F32 = 4  /* cvt.f64.f32: 1 op per conversion (chained likewise) */
} tq_pipe;

/* Run the probe of `pipe` on every SM of the current device (4 CTAs of 256
 * threads per SM, 8 independent chains per thread, `iters` x 16 instructions
 * per chain; 1 <= iters <= 2^24), four launches on a private stream, and
 * return the best of the last three as *ops_per_s (flops/s for the FMA and
 * MMA pipes, conversions/s otherwise) and its duration *ms (may be NULL).
 * Synchronous; allocates 256 bytes of device memory for the call. */
tq_status tq_pipe_rate(int pipe, int iters, double* ops_per_s, double* ms);

/* ---- per-launch profiling (CUDA events on the state's stream) ---------- */

typedef struct tq_kernel_stat {
  char name[32];      /* e.g. "apply_f64_w2", "superop_build", "fuse", "reduce" */
  uint64_t launches;
  double total_ms;    /* sum of event-timed launch durations */
  double flops;       /* algorithmic flops per launch, averaged over the launches:
                         8 per complex multiply-add of every computed group (Sec.
                         3.1) -- the dense 16^w count, except for the row-list
                         kernels ("apply_f64_sparse_w*"), which count the
                         nonzeros of the row lists they applied, read back from
                         the device after compression */
  double bytes;       /* algorithmic HBM bytes per launch, averaged over the
                         launches (one read + one write of every computed entry) */
} tq_kernel_stat;

/* Turn event timing of every kernel launch on (1) or off (0); turning it on
 * clears the statistics. */
tq_status tq_profile_enable(tq_state* s, int on);

/* Statistics since profiling was enabled, one entry per kernel kind (waits
 * for the stream). *count receives the number of kinds (<= capacity filled). */
tq_status tq_profile_read(tq_state* s, tq_kernel_stat* out, int capacity, int* count);

/* Total kernels this state has launched since creation (always counted). */
tq_status tq_launch_count(const tq_state* s, uint64_t* out);

/* ---- measurement (Sec. 3 announces measurement gates; Sec. 3.5 the
 * readout-error model; the measurement section itself is missing) -------- */

/* Selective measurement of `qubit` in the computational basis: with
 * p0 = Tr(P0 rho)/Tr(rho) (P_m = |m><m| on the qubit, FP64 reduction), the
 * outcome is 0 if u < p0, else 1 (u in [0,1) is the caller's uniform draw);
 * rho becomes P_m rho P_m / Tr(P_m rho). *outcome receives m, *probability
 * (may be NULL) its probability. Waits for the stream. */
tq_status tq_measure(tq_state* s, int qubit, double u, int* outcome, double* probability);

/* Outcome probabilities of measuring every qubit after independent
 * per-qubit readout errors: qubit q reads 1 when it is 0 with probability
 * e10[q] (prob_meas1_prep0) and reads 0 when it is 1 with e01[q]
 * (prob_meas0_prep1): the confusion matrix [[1-e10, e01], [e10, 1-e01]] on
 * every qubit, applied on the GPU to diag(rho) (renormalised in TQ_SPLIT).
 * e10, e01: n rates in [0,1]; out: 2^n doubles. Waits for the stream. */
tq_status tq_probs_readout(tq_state* s, const double* e10, const double* e01, double* out);

/* Sample `shots` outcomes of measuring every qubit: outcomes[i] = the
 * smallest x with u[i] < cdf[x] / cdf[2^n - 1], where cdf is the inclusive
 * prefix sum (FP64, fixed order) of the outcome probabilities, with the
 * readout errors e10/e01 applied first when both are given (both NULL:
 * none). u[i] in [0,1) are the caller's uniform draws. Waits for the
 * stream. */
tq_status tq_sample(tq_state* s, const double* u, int shots, const double* e10, const double* e01,
                    uint64_t* outcomes);

/* ---- host-side helpers (no GPU work; usable without a device) ----------- */

/* Matrix of a named gate: *k_out = 1 or 2, U_out receives 2^k x 2^k complex
 * (room for 16 complex = 32 doubles is enough). */
tq_status tq_gate_matrix(int gate, const double* params, int* k_out, double* U_out);

/* Kraus set of a named channel on k qubits: *m_out matrices of 2^k x 2^k
 * written to K_out, which has room for `capacity` matrices. With K_out NULL
 * only *m_out is set (count query); TQ_ERR_ARG if capacity is too small
 * (*m_out still tells the count needed). */
tq_status tq_channel_kraus(int channel, int k, const double* params, int capacity,
                           int* m_out, double* K_out);

/* Fusion plan only (the same planner tq_run_circuit uses): block_of_op[i]
 * receives the index of the block op i joins, block_width[b] the number of
 * qubits of block b (arrays of n_ops entries); *n_blocks_out the count. */
tq_status tq_plan_fusion(int n_qubits, const tq_op* ops, size_t n_ops, int max_fuse_width,
                         int precision, int* block_of_op, int* block_width,
                         size_t* n_blocks_out);

/* Structural nonzero pattern of an op's superoperator (ops on 1 or 2
 * qubits; TQ_ERR_UNSUPPORTED otherwise): *width_out = k, *nnz_out = number of
 * entries S[i][j] that may be nonzero, rows_out[i] (if not NULL, 4^k
 * entries) = bit mask of the columns j of row i. Depolarising channels give
 * their exact pattern. FP64 fused blocks of width <= 2 with at most 75%
 * nonzeros are applied from row lists (exact zeros skipped). */
tq_status tq_op_pattern(const tq_op* op, int* width_out, int* nnz_out, uint16_t* rows_out);

/* Base vec index of group g for a block whose 2k target bit positions are
 * positions[0..2k-1] (any order): g with a zero bit inserted at every target
 * position, in increasing position order. For k = 1 and positions (q, q+n)
 * this is the index s_i of Sec. 3.1. */
uint64_t tq_group_base(uint64_t g, const int* positions, int n_positions);

const char* tq_status_string(int status);

/* Library version string. */
const char* tq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TANQ_H */
