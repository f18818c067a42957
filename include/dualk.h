/*
 * dualk -- C ABI of the GB300 (sm_103a) quantum-classical dual-kernel engine.
 *
 * Paper: "Scalable Tensor Network Simulation for Quantum-Classical Dual Kernel"
 * (arXiv 2602.01330). The library computes, on one GPU,
 *
 *   K_q(x_i, x_j) = |<psi(x_i)|psi(x_j)>|^2                         (§II-C, Eqs. 6-10)
 *   K_c(x_i, x_j) = exp(-gamma ||x_i - x_j||^2)                       (§II-B, Eq. 3)
 *   K(x_i, x_j)   = w K_q + (1 - w) K_c                               (§II-D, Eq. 11)
 *
 * with |psi(x)> held as a matrix product state (MPS) and K_q evaluated by
 * contracting the compute-uncompute overlap network as a chain of transfer
 * matrices, E <- sum_s A_s(x_i)^dagger E A_s(x_j), tile by tile over blocks of
 * (row, column) sample pairs (§II-C: exact tensor-network contraction; §II-D:
 * blockwise construction of the kernel matrix).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named x, mps, log_norm, bond_dims, k_out, kq_out, kc_out, logkq_out
 *   are DEVICE pointers, allocated and owned by the caller. The library never
 *   allocates, frees or keeps them. `stream` is a cudaStream_t passed as void*
 *   (NULL = the legacy default stream). Every call is asynchronous on `stream`;
 *   inputs must stay valid and outputs untouched until the stream reaches the call.
 * - Features x are float32, row-major m x n (sample-major): x[i*n + f].
 * - MPS layout (written by dk_mps_build, read by the Gram calls). Every bond of the
 *   ZZ-chain MPS carries a copy of the computational value of the qubit to its left, so
 *   with bond positions ordered as b = t*h + j (t = that bit, h = chi_max/2) the site
 *   tensor A_s[l][b] vanishes unless b lies in block s. Only the non-zero half is stored,
 *   site-major:
 *       A[k][i][s][j][l],  k < n sites, i < m samples, s in {0,1},
 *       j < h (right bond position s*h + j), l < chi_max (left bond position),
 *   l fastest: element (k,i,s,j,l) sits at index (((k*m + i)*2 + s)*h + j)*chi_max + l,
 *   complex64 (float re, float im) for DK_C64 or complex128 for DK_C128, chi_max^2
 *   complex numbers per sample and site. At the last site the right bond is 1 and both
 *   s use j = 0. Unused bond positions are zero. Base pointers must be 16-byte aligned
 *   (cudaMalloc / torch allocations are).
 * - Errors: every call returns a dk_status. Argument errors are detected on the
 *   host before anything is launched (DK_ERR_ARG, DK_ERR_UNSUPPORTED). A failing
 *   CUDA launch returns DK_ERR_CUDA. A device-side wait that exceeds its bound
 *   (about two seconds) makes the kernel record DK_ERR_TIMEOUT in the context's
 *   status word and return without finishing; an index out of range in a device-side
 *   list (SVM calls) is skipped and recorded the same way; dk_sync_status reads it. No
 *   call aborts, asserts or traps.
 */
#ifndef DUALK_H
#define DUALK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DK_OK = 0,
  DK_ERR_ARG = 1,          /* invalid argument: NULL pointer, bad size, misaligned pointer */
  DK_ERR_UNSUPPORTED = 2,  /* combination of chi_max / dtype / precision not built */
  DK_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
  DK_ERR_TIMEOUT = 4,      /* a device-side wait exceeded its bound (read via dk_sync_status) */
  DK_ERR_WORKSPACE = 5,    /* caller-provided workspace too small */
  DK_ERR_NO_DEVICE = 6     /* no usable sm_100-family device */
} dk_status;

/* Buffer formats of an MPS. DK_C64 / DK_C128: the site tensors (layout above) in complex64 /
 * complex128. DK_SPLIT_BF16: the split-BF16 tensor-core operands of a bond-32 complex64 MPS,
 * written by dk_mps_split32 and read by the DK_PREC_BF16X3 Gram calls (layout there). */
typedef enum { DK_C64 = 0, DK_C128 = 1, DK_SPLIT_BF16 = 2 } dk_dtype;

/* Arithmetic of the transfer contraction. F32: complex64 tensors, FP32 FMA on CUDA
 * cores (chi_max 4, 8, 32). F64: complex128 tensors, FP64 (chi_max 4). BF16X3: complex64
 * tensors at chi_max 32 on tensor cores, each FP32 operand split into two BF16 halves
 * (hi + lo) and each product formed as hi.hi + hi.lo + lo.hi with FP32 accumulation
 * (about 16 significant bits per product); the Gram calls also take the operands already
 * split (dtype DK_SPLIT_BF16, dk_mps_split32), which is the faster form. */
typedef enum {
  DK_PREC_F32 = 0,
  DK_PREC_F64 = 1,
  DK_PREC_BF16X3 = 2
} dk_precision;

/* Kernels of the split-BF16 block-statevector Gram (dk_set_block_gram_form). */
typedef enum {
  DK_BLOCK_TCGEN05 = 0,  /* tcgen05.mma, TMEM accumulators, TMA loads (default) */
  DK_BLOCK_MMA_SYNC = 1  /* warp-level mma.sync m16n8k16 */
} dk_block_form;

typedef struct dk_ctx dk_ctx;

/* Feature map U(x) of §II-C (Eq. 6). The paper's circuit figure is not in its text;
 * the map built here is the ZZ chain: per repetition, H on every qubit, then
 * RZ(angle_scale * x_i) on qubit i, then (if entangle) RZZ(2 (pi - x_i)(pi - x_{i+1}))
 * on every neighbouring pair of the open chain; the same x is re-uploaded by every
 * repetition. With block = b >= 1 the entanglers are block-structured (the block product
 * state form §II-C describes): the qubits form blocks of b consecutive qubits (the last
 * may be shorter) and only pairs inside a block get an RZZ, so the state is a product of
 * the blocks' own chain states and K_q a product of per-block kernels. */
typedef struct {
  int reps;           /* repetitions, 1..5 */
  float angle_scale;  /* RZ angle = angle_scale * x_i (2 for the ZZ-chain map) */
  int entangle;       /* 1: RZZ chain applied; 0: product state */
  int chi_max;        /* stored bond dimension: 4, 8, 16 or 32, and >= 2^reps */
  int qr_prec;        /* arithmetic of the left-canonical QR sweep for complex64 output at
                         chi_max 4: DK_PREC_F32 (0, default) or DK_PREC_F64. complex128
                         output and wider bonds always use FP64. */
  int block;          /* 0: one block (the whole chain); b >= 1: entanglers only inside
                         blocks of b consecutive qubits (b = 1: none, b >= n: the chain) */
} dk_fmap;

/* Create a context on `device` (sets it current on the calling thread). The context
 * holds the device status word and cached launch parameters; it never owns user
 * buffers. Returns DK_ERR_NO_DEVICE if the device is not compute capability 10.x.
 * Calls on a context must be made with its device current. Every launch sets its kernel's
 * shared-memory opt-in itself (the setting is per device), so contexts on several devices
 * of one process are possible; multi-GPU runs here use one process per GPU, and only that
 * arrangement has been run. */
dk_status dk_create(dk_ctx** out, int device);
void dk_destroy(dk_ctx* ctx);
const char* dk_error_string(dk_status status);

/* Wait for `stream`, then return and clear the device status word (DK_OK if no
 * kernel recorded an error since the last call): DK_ERR_TIMEOUT for an expired bounded
 * wait, else DK_ERR_ARG for an out-of-range index found in a device array (SVM calls). */
dk_status dk_sync_status(dk_ctx* ctx, void* stream);

/* Failure-detection self test: launches a kernel whose wait can never be satisfied (an
 * mbarrier that nothing arrives on), bounded by limit_ns (1 .. 2e9). The kernel gives up,
 * records DK_ERR_TIMEOUT in the status word and returns, so the next dk_sync_status
 * reports DK_ERR_TIMEOUT and the context stays usable. This exercises the same bounded
 * wait and status path as the Gram kernels without faulting or hanging the GPU.
 * Errors: DK_ERR_ARG for NULL ctx or limit_ns outside 1 .. 2e9; DK_ERR_CUDA. */
dk_status dk_selftest_wait_timeout(dk_ctx* ctx, unsigned long long limit_ns, void* stream);

/* Bytes of an MPS buffer for m samples, n sites, padded bond chi_max (DK_SPLIT_BF16:
 * chi_max 32 only, 10240 bytes per sample and site; 0 for other bonds). */
size_t dk_mps_bytes(int m, int n, int chi_max, dk_dtype dtype);

/* Split-BF16 operands of a bond-32 complex64 MPS for the DK_PREC_BF16X3 Gram calls
 * (§II-C, Eqs. 8-10 on tensor cores). For every site k and sample i the four 16 x 16
 * blocks A_s[t] (s, t in {0, 1}) are written as the real operand X = [Re A^T | Im A^T]
 * (16 rows of 32 values; row p holds Re A[l][p] for l < 16, then Im A[l][p]), each value v
 * split into BF16 hi = round(v) and lo = round(v - hi), so that the Gram kernels copy them
 * to shared memory as they are instead of splitting them again for every tile:
 *   ops[((k*m + i)*4 + 2*s + t)*2 + plane][p][c],  plane 0 = hi, 1 = lo, p < 16, c < 40,
 * BF16 values, c >= 32 zero (row padding that spreads the tensor-core operand reads over
 * the shared-memory banks): 10240 bytes per sample and site, dk_mps_bytes(m, n, 32,
 * DK_SPLIT_BF16) in all. The Gram calls take `ops` in place of the MPS with dtype
 * DK_SPLIT_BF16, prec DK_PREC_BF16X3 and chi_max 32, and give bit for bit the results of
 * the same call on the complex64 MPS; the self-norms (dk_self_overlap, prec BF16X3) and
 * the refinement (dk_gram_refine) keep reading the complex64 MPS.
 *   mps: device, dk_mps_build layout, complex64, chi_max 32, m samples, n sites;
 *   ops: device, ops_bytes >= dk_mps_bytes(m, n, 32, DK_SPLIT_BF16), 16-byte aligned.
 * Errors: DK_ERR_ARG (NULL or misaligned pointers, m or n < 1), DK_ERR_WORKSPACE (ops_bytes
 *         too small), DK_ERR_CUDA. */
dk_status dk_mps_split32(dk_ctx* ctx, const void* mps, int m, int n, void* ops, size_t ops_bytes, void* stream);

/* Scratch bytes the build, Gram and rows calls (dk_mps_build, dk_gram_tile,
 * dk_dual_kernel_rows, dk_gram_sweep) need for (n, chi_max, dtype, prec): always 0. Every
 * kernel of these calls keeps its working state in registers and shared memory and writes
 * only the caller's outputs, so they take no workspace argument; the query exists for
 * callers that size a workspace per call. Returns (size_t)-1 for a combination no kernel
 * supports (chi_max / dtype / prec as dk_gram_tile), so it also serves as a capability
 * check. The block-statevector calls, which do need scratch in one form, have their own
 * queries (dk_block_states_workspace_bytes, dk_gram_blocks_workspace_bytes). */
size_t dk_workspace_bytes(int n, int chi_max, dk_dtype dtype, dk_precision prec);

/* |psi(x_i)> = U(x_i)|0>^n as an MPS (§II-C, Eq. 6), for i < m.
 *
 * Exact construction: every RZZ layer is a diagonal bond-2 operator, so after r
 * repetitions the state is an MPS of bond 2^r whose site tensors have a closed form
 * in (x_{k-1}, x_k). Each sample's chain is then brought to left-canonical form by QR,
 * one bond block at a time (Gram-Schmidt with re-orthogonalisation at bond 4, Householder
 * for wider bonds), normalised, and rounded to `dtype`. The QR arithmetic is FP64, except
 * for complex64 output at chi_max 4 with fm->qr_prec = DK_PREC_F32 (the default), where it
 * is FP32; no bond is truncated in either case.
 *   x          m x n float32 features (device)
 *   fm         feature map (host pointer)
 *   mps        dk_mps_bytes(m, n, fm->chi_max, dtype) bytes (device, written)
 *   bond_dims  n + 1 int32 (device, written, may be NULL): number of non-zero left-bond
 *              positions of site k (1, 2, 4, ... up to 2^reps), and 1 at index n. With
 *              block >= 1 the stored bond at a block boundary keeps the chain's size
 *              (its exact rank is 1; the extra positions hold rounding-level columns).
 *   log_norm   m floats (device, written, may be NULL): ln |<psi~_i|psi~_i>| of the
 *              rounded tensors, evaluated by the same transfer arithmetic as the Gram
 *              calls; passing it to them normalises K_q so that K_q(x, x) = 1.
 * Errors: DK_ERR_ARG (m < 1, n < 1, NULL x/mps/fm, reps outside 1..5, qr_prec neither
 *         DK_PREC_F32 nor DK_PREC_F64, block < 0, misaligned mps),
 *         DK_ERR_UNSUPPORTED (chi_max not in {4, 8, 16, 32} or below 2^reps; log_norm
 *         requested for a chi_max / dtype without a Gram kernel: complex64 has chi_max 4,
 *         8 and 32, complex128 chi_max 4). */
dk_status dk_mps_build(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm,
                       dk_dtype dtype, void* mps, int32_t* bond_dims, float* log_norm,
                       void* stream);

/* Entanglers inside a block for dk_mps_build_blocks. */
#define DK_ENT_CHAIN 0 /* RZZ on neighbouring pairs (i, i+1) of the block */
#define DK_ENT_FULL 1  /* RZZ(2 (pi - x_i)(pi - x_j)) on every pair i < j of the block */

/* MPS of a block-structured feature map (§II-C: entanglers only inside blocks of b
 * consecutive qubits, dk_fmap.block) from its block statevectors, with SVD truncation.
 * Per sample and block (b <= 12 qubits): the dense 2^b statevector of the block in FP64
 * (per repetition H on every qubit, RZ(angle_scale x_q), then the RZZ of every entangled
 * pair), then a left-to-right sweep of singular value decompositions (one-sided Jacobi in
 * FP64): at each cut the singular values s > cutoff * s_0 are kept, at most chi_max / 2 of
 * them, rescaled to the norm of the whole spectrum, and the discarded squared weight is
 * accumulated. The bond at a block boundary is 1. With DK_ENT_FULL the exact bond inside a
 * block reaches 2^min(q, b - q) at the cut after q qubits, beyond the 2^reps of the chain.
 *   x          m x n float32 features (device)
 *   fm         reps 1..5, angle_scale, entangle (0: product state), chi_max 4, 8, 16 or 32
 *              (stored width; kept bond <= chi_max / 2), block 1..12 (0: one block, n <= 12);
 *              qr_prec is ignored (FP64 throughout)
 *   entangler  DK_ENT_CHAIN or DK_ENT_FULL
 *   cutoff     relative singular value cutoff, 0 <= cutoff < 1 (1e-10 drops only numerical
 *              zeros)
 *   mps        dk_mps_bytes(m, n, chi_max, dtype) bytes (device, written). Layout as
 *              dk_mps_build: a site tensor B_s[a][j] (left bond a, right bond j < chi_max/2)
 *              is stored at block s, column j, left positions a and chi_max/2 + a, so the
 *              Gram calls for chi_max contract the general MPS unchanged.
 *   bond_dims  n + 1 int32 (device, written, may be NULL): kept bond left of each site, the
 *              largest over the samples (1 at block starts and at index n)
 *   log_norm   m floats (device, written, may be NULL): as dk_mps_build
 *   discarded  m floats (device, written, may be NULL): discarded squared weight of each
 *              sample summed over its cuts (0 when nothing was truncated)
 * One CTA per sample; the call allocates nothing.
 * Errors: DK_ERR_ARG (NULL ctx/x/fm/mps, m or n < 1, reps outside 1..5, unknown entangler,
 *         cutoff outside [0, 1), dtype, misaligned mps), DK_ERR_UNSUPPORTED (block < 0 or a
 *         block above 12 qubits, chi_max not in {4, 8, 16, 32}, log_norm for a chi_max /
 *         dtype without a Gram kernel), DK_ERR_CUDA. */
dk_status dk_mps_build_blocks(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, int entangler,
                              double cutoff, dk_dtype dtype, void* mps, int32_t* bond_dims, float* log_norm,
                              float* discarded, void* stream);

/* One item of a feature-dimension sweep: the symmetric Gram of one MPS batch. */
typedef struct {
  const void* mps;        /* m samples, n sites (dk_mps_build layout, chi_max / dtype of the call) */
  const float* log_norm;  /* m ln-norms in the arithmetic of the call's precision */
  const float* x;         /* m x n features (needed for K_c: kc, or k with w != 1) */
  float* k;               /* m x m outputs with row stride ld, any may be NULL but not all */
  float* kq;
  float* kc;
  float* logkq;
  long long ld;
  int m, n;
  int tile_shape;         /* 0: built-in tile shape; 1..dk_gram_config_count: a fixed one */
} dk_sweep_item;

/* The symmetric Gram matrices of a feature-dimension sweep (§II-D: a kernel matrix for
 * every qubit count of a study, each filled block by block), each item as
 * dk_gram_tile over all its samples with gamma = 1/n, mix weight w and precision prec,
 * followed, for complex64 items in F32 or BF16X3 with kq or logkq, by dk_gram_refine with
 * tau = DK_REFINE_TAU (declared below) and the workspace ws / ws_bytes (NULL / 0: no
 * workspace; otherwise dk_gram_refine_workspace_bytes(m, m) bytes for the largest item m,
 * caller-owned, reused by the items one after the other), issued in order on `stream`.
 * graph = 0: the launches are issued directly.
 * graph = 1: the launches are recorded once into a CUDA graph that the context keeps
 *   (keyed by the bytes of the item array and the other arguments, pointers and ws included) and
 *   replayed by every later call with the same key: one graph launch for the whole sweep.
 *   The first call with a new key also computes the results (eagerly, before recording).
 *   A replay reads the items' current buffer contents, so inputs may change between calls;
 *   buffers must stay allocated while the context may replay them. At most 16 graphs are
 *   kept (the oldest is destroyed); dk_destroy releases them. Needs a non-NULL stream.
 * Errors: DK_ERR_ARG (NULL ctx/items, n_items < 1, an item with NULL mps or log_norm, m or
 *         n < 1, no output, ld < m, tile_shape out of range; graph with the NULL stream),
 *         DK_ERR_UNSUPPORTED for dtype DK_SPLIT_BF16 (the refinement reads complex64 site
 *         tensors), and those of dk_gram_tile; DK_ERR_CUDA if recording or instantiation fails. */
dk_status dk_gram_sweep(dk_ctx* ctx, const dk_sweep_item* items, int n_items, int chi_max, dk_dtype dtype,
                        dk_precision prec, float w, int graph, void* ws, size_t ws_bytes, void* stream);

/* Block statevectors of a block-structured feature map (§II-C: entanglers only inside
 * blocks of b consecutive qubits, chain or all-to-all as for dk_mps_build_blocks). The state
 * is the Kronecker product of its blocks' states, so the overlap of Eq. 9 factorises over
 * the blocks and dk_gram_blocks contracts it exactly, block by block, with no MPS bond.
 * Bytes: nb * m * dpad * 8, nb = ceil(n / b) blocks, dpad = max(2^b, 16) complex64
 * amplitudes per (block, sample); 0 if block is outside 0..12 (0: one block, n <= 12). */
size_t dk_block_states_bytes(int m, int n, int block);

/*   x         m x n float32 features (device)
 *   fm        reps 1..5, angle_scale, entangle (0: product state), block (see above);
 *             chi_max and qr_prec are ignored
 *   entangler DK_ENT_CHAIN or DK_ENT_FULL
 *   prec      DK_PREC_F32: states for the FP32 CUDA-core Gram; DK_PREC_BF16X3: for the
 *             split-BF16 tensor-core Gram (pass the same precision to dk_gram_blocks)
 *   states    dk_block_states_bytes(m, n, fm->block) bytes (device, written), layout
 *             [block][sample][...] of dpad amplitudes (qubit 0 of the block most
 *             significant), computed in FP64 and rounded once: F32 as complex64 values;
 *             BF16X3 as split values v ~ hi + lo, per chunk of 16 amplitudes one
 *             128-byte row of four BF16 planes [hi(re) | hi(im) | lo(re) | lo(im)] of 16
 *             values each; zeros beyond 2^b and beyond the 2^(n mod b) amplitudes of a short
 *             last block
 *   log_norm  m floats (device, written, may be NULL): ln|<psi~_i|psi~_i>| of the rounded
 *             states by the arithmetic of dk_gram_blocks in `prec` (for BF16X3 the diagonal
 *             tiles of that Gram, in the context's dk_set_block_gram_form form), so that
 *             K_q(x, x) = 1 exactly
 *   ws        caller-owned device scratch of at least ws_bytes =
 *             dk_block_states_workspace_bytes(ctx, m, n, fm->block, prec) bytes, 16-byte
 *             aligned (the tcgen05 form of the BF16X3 self-norms keeps one value per block
 *             and sample there); may be NULL when that size is 0 or log_norm is NULL. Its
 *             contents are scratch: nothing is read from it before it is written.
 * Errors: DK_ERR_ARG (NULL pointers, m or n < 1, reps, entangler, misaligned states),
 *         DK_ERR_UNSUPPORTED (block outside 0..12 or above 12 qubits, m > 65535, more than
 *         6144 blocks, prec neither F32 nor BF16X3), DK_ERR_WORKSPACE (ws NULL, misaligned or
 *         smaller than the query's size), DK_ERR_CUDA. */
dk_status dk_block_states(dk_ctx* ctx, const float* x, int m, int n, const dk_fmap* fm, int entangler,
                          dk_precision prec, void* states, float* log_norm, void* ws, size_t ws_bytes, void* stream);

/* Scratch bytes dk_block_states needs for these arguments on this context (it depends on
 * dk_set_block_gram_form): nb * m * 4 rounded up to 256 for DK_PREC_BF16X3 in the tcgen05
 * form, else 0; 0 also for arguments the call would reject. */
size_t dk_block_states_workspace_bytes(dk_ctx* ctx, int m, int n, int block, dk_precision prec);

/* A block of the Gram matrix of a block-structured map from block statevectors, outputs
 * and epilogue as dk_gram_tile (§II-C Eqs. 8-10 factorised over blocks; §II-B Eq. 3;
 * §II-D Eq. 11): for each pair, a = prod_B <psi_B(x_i)|psi_B(x_j)> with each factor a
 * complex dot product of 2^b amplitudes — prec DK_PREC_F32: FP32 FMAs on CUDA cores;
 * DK_PREC_BF16X3: split-BF16 tensor-core products with FP32 accumulation (|dK| ~ 1e-5,
 * the 1e-4 mixed-precision class; tcgen05 or mma.sync kernels as dk_set_block_gram_form
 * selects) — and ln|a| accumulated as a sum of log2 |factor|^2
 * (never underflows); log K_q = 2 ln|a| - ln N_i - ln N_j, K_q,
 * K_c = exp(-gamma ||x_i - x_j||^2), K = w K_q + (1 - w) K_c.
 *   states_rows / states_cols  dk_block_states output for m_rows / m_cols samples, same n
 *                              and block; lnorm_rows / lnorm_cols their log_norm
 *   x_rows / x_cols            features (needed for K_c: kc_out, or k_out with w != 1)
 *   k_out, kq_out, kc_out, logkq_out  nrows x ncols float32 (device, any may be NULL, not
 *                              all), row stride ld; symmetric (rows == cols, same range)
 *                              computes each unordered pair once and writes both entries
 *   ws, ws_bytes               caller-owned device scratch, 16-byte aligned, of at least
 *                              dk_gram_blocks_workspace_bytes(ctx, n, block, nrows, ncols,
 *                              prec, symmetric, K_c needed) bytes: the tcgen05 form of
 *                              DK_PREC_BF16X3 keeps the RBF distances there (nrows * ncols * 4
 *                              bytes when K_c is needed) and, for a rectangular block split
 *                              over its blocks, the partial sums (up to 8 * nrows * ncols * 4
 *                              bytes); NULL when that size is 0. Nothing is read from it
 *                              before it is written. The library allocates nothing.
 * Errors: DK_ERR_ARG (NULL inputs, ranges outside the sample counts, ld < ncols, no
 *         output, symmetric with different rows and columns, K_c needed without x),
 *         DK_ERR_UNSUPPORTED (block, prec neither F32 nor BF16X3), DK_ERR_WORKSPACE (ws
 *         NULL, misaligned or smaller than needed), DK_ERR_CUDA. */
dk_status dk_gram_blocks(dk_ctx* ctx, const void* states_rows, int m_rows, const void* states_cols, int m_cols,
                         int n, int block, int row0, int nrows, int col0, int ncols, const float* lnorm_rows,
                         const float* lnorm_cols, const float* x_rows, const float* x_cols, float gamma, float w,
                         dk_precision prec, float* k_out, float* kq_out, float* kc_out, float* logkq_out,
                         long long ld, int symmetric, void* ws, size_t ws_bytes, void* stream);

/* Scratch bytes of a dk_gram_blocks call with these sizes on this context (the plan depends
 * on the SM count and dk_set_block_gram_form); with_kc: 1 when K_c is needed (kc_out, or
 * k_out with w != 1). 0 for DK_PREC_F32, for the mma.sync form, and for arguments the call
 * would reject. */
size_t dk_gram_blocks_workspace_bytes(dk_ctx* ctx, int n, int block, int nrows, int ncols, dk_precision prec,
                                      int symmetric, int with_kc);

/* Refinement of the large values of a block written by dk_gram_blocks (§II-C Eqs. 7-10,
 * factorised over the blocks; §II-D Eq. 11). The Gram kernels form each block's overlap as
 * an FP32 (or split-BF16) dot product of 2^b amplitudes and sum the logs over the blocks;
 * on K_q of order one at n = 784 in blocks of 10 that leaves about 5e-5 (FP32) and 4e-4
 * (split BF16). This call recomputes every entry with K_q > tau (log K_q > ln tau when
 * kq_out is NULL; not the symmetric diagonal): for every block the overlap and both
 * self-overlaps of the stored amplitudes with exact products and compensated (Dot2)
 * sums, the lanes of a warp added in FP64, log K_q = sum_B [log |<a_B|b_B>|^2 - log
 * <a_B|a_B> - log <b_B|b_B>] in FP64; then K_q, log K_q and K as dk_gram_refine does. One
 * warp per refined entry: the cost is proportional to the entries above tau.
 *   Arguments as for the dk_gram_blocks call that wrote the block (states, sizes, n, block,
 *   prec, range, x, gamma, w, outputs, ld, symmetric); tau in (0, 1).
 * Errors: DK_ERR_ARG (as dk_gram_refine), DK_ERR_UNSUPPORTED (block, prec), DK_ERR_CUDA. */
dk_status dk_gram_blocks_refine(dk_ctx* ctx, const void* states_rows, int m_rows, const void* states_cols, int m_cols,
                                int n, int block, dk_precision prec, int row0, int nrows, int col0, int ncols,
                                const float* x_rows, const float* x_cols, float gamma, float w, float tau,
                                float* k_out, float* kq_out, float* kc_out, float* logkq_out, long long ld,
                                int symmetric, void* stream);

/* Kernels the context uses for DK_PREC_BF16X3 block states' self-norms and block Grams:
 * DK_BLOCK_TCGEN05 (default; 128 x 128 or 128 x 64 pair tiles, one CTA per SM, tcgen05.mma
 * from TMA-loaded shared memory into tensor-memory accumulators) or DK_BLOCK_MMA_SYNC. Both
 * read the same states and agree to rounding; K_q(x, x) = 1 exactly holds when the states'
 * log_norm and the Gram come from the same form.
 * Errors: DK_ERR_ARG (NULL ctx, unknown form). */
dk_status dk_set_block_gram_form(dk_ctx* ctx, int form);

/* ln|<psi~_i|psi~_i>| of the stored (rounded) MPS of m samples, computed with the
 * arithmetic of precision `prec`, so that a Gram call with the same precision and these
 * normalisers gives K_q(x, x) = 1 exactly (§II-C, Eq. 7 for unit-norm states).
 * dk_mps_build already writes the F32 (complex64) / F64 (complex128) normalisers; this
 * call provides them for another precision (BF16X3).
 *   mps: device MPS (dk_mps_build layout); log_norm: m floats (device, written).
 * Errors: DK_ERR_ARG (NULL pointers, m or n < 1), DK_ERR_UNSUPPORTED (no kernel for
 *         chi_max / dtype / prec). */
dk_status dk_self_overlap(dk_ctx* ctx, const void* mps, int m, int n, int chi_max, dk_dtype dtype,
                          dk_precision prec, float* log_norm, void* stream);

/* One block of the Gram matrix (§II-D: block (i:i+B, j:j+B) contracted by a GPU
 * worker), with the RBF kernel and the mix fused into the epilogue.
 *
 * Rows are samples row0 .. row0+nrows-1 of the MPS `mps_rows` (which holds m_rows
 * samples) and columns are samples col0 .. col0+ncols-1 of `mps_cols` (m_cols
 * samples); both were built with the same n, chi_max and dtype. For each pair,
 *   a    = <psi(x_i)|psi(x_j)>  by the transfer chain with per-site power-of-two
 *          rescaling (never underflows),
 *   logkq = 2 ln|a| - log_norm_rows[i] - log_norm_cols[j]  (log_norm NULL => 0),
 *   kq   = exp(logkq),  kc = exp(-gamma ||x_i - x_j||^2),  k = w kq + (1 - w) kc.
 * Outputs (each may be NULL; all float32, device) are written at
 * out[(i - row0) * ld + (j - col0)].
 * symmetric = 1 requires mps_rows == mps_cols, row0 == col0, nrows == ncols; each
 * unordered pair is then contracted once and written to both (i,j) and (j,i).
 *   x_rows / x_cols: the m_rows x n / m_cols x n features the MPS were built from;
 *   needed only when k_out or kc_out is requested.
 * dtype DK_SPLIT_BF16 (prec DK_PREC_BF16X3, chi_max 32): mps_rows / mps_cols are the
 * split operands dk_mps_split32 wrote from the MPS; log_norm_* still come from the MPS
 * (dk_self_overlap with prec BF16X3).
 * Errors: DK_ERR_ARG (ranges outside the MPS, ld < ncols, bad symmetric request,
 *         NULL x when k/kc requested), DK_ERR_UNSUPPORTED (precision/dtype/chi). */
dk_status dk_gram_tile(dk_ctx* ctx,
                       const void* mps_rows, int m_rows, const void* mps_cols, int m_cols,
                       int n, int chi_max, dk_dtype dtype,
                       int row0, int nrows, int col0, int ncols,
                       const float* log_norm_rows, const float* log_norm_cols,
                       const float* x_rows, const float* x_cols,
                       float gamma, float w, dk_precision prec,
                       float* k_out, float* kq_out, float* kc_out, float* logkq_out,
                       int64_t ld, int symmetric, void* stream);

/* Dual-kernel rows for prediction (§II-B, Eq. 5 needs K(x_i, x) for every training
 * sample x_i): the b x m block K(test, train), row-major with leading dimension m.
 * Same arithmetic and output conventions as dk_gram_tile with rows = the b test
 * samples and columns = the m training samples. */
dk_status dk_dual_kernel_rows(dk_ctx* ctx,
                              const void* mps_test, const float* x_test, const float* log_norm_test, int b,
                              const void* mps_train, const float* x_train, const float* log_norm_train, int m,
                              int n, int chi_max, dk_dtype dtype, float gamma, float w,
                              dk_precision prec,
                              float* k_out, float* kq_out, float* kc_out, float* logkq_out,
                              void* stream);

/* Threshold the sweep call and the Python binding use for dk_gram_refine. */
#define DK_REFINE_TAU 0.02f

/* Refinement of the large values of a block written by dk_gram_tile or dk_dual_kernel_rows
 * (§II-C Eqs. 7-10; §II-D Eq. 11). The FP32 transfer chain rounds E at every site, and the
 * rounding of its dominant direction adds up over the n sites like a random walk: a K_q of
 * order one comes out with a relative error of about sqrt(n) * 6 u (7e-6 at n = 784, bond 4;
 * 1e-5 at bond 32 and n = 256; split-BF16 products, about 16 significant bits: 1e-3), small
 * values with the same relative error. This call recomputes every entry of the block with
 * K_q > tau (log K_q > ln tau when kq_out is NULL): the amplitude and both self-overlaps by
 * the same chain on the same complex64 tensors, with E kept as double-word FP32 sums hi + lo
 * (error-free products and additions, about 44 bits), and writes K_q, log K_q and K (K_c
 * read from kc_out or recomputed as the Gram call forms it). Other entries keep their bits;
 * the diagonal of a symmetric block (exactly 1) is not touched. With tau = 0.02 the FP32
 * paths stay within |dK| <= 1e-6 and the split-BF16 path within 1e-4 of the exact values.
 *   The block arguments are those of the Gram call that wrote it: rows [row0, row0 + nrows)
 *   of mps_rows x columns [col0, col0 + ncols) of mps_cols (dk_mps_build layout, complex64,
 *   chi_max 4, 8 or 32), outputs with row stride ld; symmetric as for dk_gram_tile (only
 *   j > i is examined, both entries written). x_rows / x_cols, gamma, w: as for that call
 *   (x needed only when k_out is given with w != 1 and kc_out is NULL).
 *   tau in (0, 1).
 *   ws, ws_bytes  optional caller-owned device scratch of dk_gram_refine_workspace_bytes(
 *                 m_rows, m_cols) bytes, 16-byte aligned: with it the pass first marks the
 *                 samples that entries above tau need and computes each of their ln-norms
 *                 once (three extra launches: a clear, a scan, the norms), so an entry costs
 *                 one chain instead of three — the choice when many entries exceed tau; NULL
 *                 (ws_bytes ignored): each entry computes both of its norms. Both give the
 *                 same values. Nothing is read from ws before it is written.
 * Bond 4 / 8: one thread per refined entry (queued per warp); bond 32: one warp per entry
 * (chains of about 1e9 operations each), so the cost is proportional to the number of
 * entries above tau: nothing but reads of the block when there are none.
 * Errors: DK_ERR_ARG (NULL pointers, ranges, ld < ncols, neither kq_out nor logkq_out, tau
 *         outside (0, 1), symmetric with different rows and columns, x missing when K_c has
 *         to be recomputed, misaligned MPS), DK_ERR_UNSUPPORTED (complex128, other chi_max),
 *         DK_ERR_WORKSPACE (ws too small or misaligned), DK_ERR_CUDA. */
dk_status dk_gram_refine(dk_ctx* ctx, const void* mps_rows, int m_rows, const void* mps_cols, int m_cols, int n,
                         int chi_max, dk_dtype dtype, int row0, int nrows, int col0, int ncols, const float* x_rows,
                         const float* x_cols, float gamma, float w, float tau, float* k_out, float* kq_out,
                         float* kc_out, float* logkq_out, long long ld, int symmetric, void* ws, size_t ws_bytes,
                         void* stream);

/* Scratch bytes of dk_gram_refine's once-per-sample ln-norms: (m_rows + m_cols) flags and
 * doubles, each array rounded up to 256 bytes; 0 for a size below 1. */
size_t dk_gram_refine_workspace_bytes(int m_rows, int m_cols);

/* Tile shapes of the Gram kernels (the blocks of §II-D, sized for one GB300 SM).
 * Shape 0 is the built-in choice; shapes 1..dk_gram_config_count(dtype, chi_max) can be
 * selected per context with dk_set_gram_config, e.g. by an autotuner that times them on
 * the caller's workload. dk_gram_config_info reports a shape's tile (row samples x
 * column samples) and threads per CTA; any pointer may be NULL.
 * Errors: DK_ERR_ARG for an unknown id or NULL ctx. */
int dk_gram_config_count(dk_dtype dtype, int chi_max);
dk_status dk_gram_config_info(dk_dtype dtype, int chi_max, int id, int* tile_rows, int* tile_cols,
                              int* threads);
dk_status dk_set_gram_config(dk_ctx* ctx, int id);

/* Concentration diagnostics of a kernel block (§I: exponential concentration of quantum
 * kernels; the conclusion's kernel diagnostics): over the entries of an nrows x ncols block
 * (symmetric = 1: the strict upper triangle of a square Gram, each pair of distinct samples
 * once), in FP64:
 *   out[0] = entries of kq counted, out[1] = sum K_q, out[2] = sum K_q^2,
 *   out[3] = entries of logkq with a finite value, out[4] = sum log K_q, out[5] = sum (log K_q)^2,
 *   out[6] = mean K_q, out[7] = variance of K_q, out[8] = mean log K_q, out[9] = variance of
 *   log K_q (population variances from the sums; NaN when no entry was counted)
 * (log K_q stays informative where K_q underflows to 0).
 *   kq, logkq  float32 blocks with row stride ld >= ncols (device); either may be NULL (its
 *              three sums stay 0 and its mean and variance are NaN)
 *   out        10 doubles (device, written; cleared by the call first)
 * Errors: DK_ERR_ARG (NULL ctx / out, both kq and logkq NULL, nrows or ncols < 1, ld < ncols,
 *         symmetric with nrows != ncols), DK_ERR_CUDA. */
dk_status dk_gram_stats(dk_ctx* ctx, const float* kq, const float* logkq, long long ld, int nrows, int ncols,
                        int symmetric, double* out, void* stream);

/* Largest feature count p of the PCA calls below. */
#define DK_PCA_MAX_FEATURES 4096

/* Bytes of the caller-provided workspace of dk_pca_fit for p features (2 p^2 floats and a
 * table of p / 2 rotations, 256-byte aligned parts); 0 for p outside 2..DK_PCA_MAX_FEATURES. */
size_t dk_pca_workspace_bytes(int p);

/* Data pre-processing of §II-A, fit on the training rows: standardisation (zero mean, unit
 * population variance per feature; scale 1 for a constant feature) and PCA (the eigenvectors
 * of the covariance Z^T Z / (m - 1) of the standardised rows, by parallel cyclic Jacobi in
 * FP32, `sweeps` sweeps of p - 1 rounds each, no host synchronisation).
 *   x            m x p float32, row-major (device), m >= 2
 *   k            components kept, 1..p
 *   workspace    dk_pca_workspace_bytes(p) bytes (device, 256-byte aligned), overwritten
 *   mean, scale  p floats each (device, written)
 *   components   k x p floats (device, written): orthonormal rows in order of decreasing
 *                eigenvalue, each with its entry of largest magnitude positive
 *   eigenvalues  k floats (device, written)
 *   off_norm     1 float (device, written, may be NULL): sqrt(off-diagonal / total sum of
 *                squares) of the rotated covariance after the last sweep (about 1e-7 when
 *                the sweeps sufficed)
 * Errors: DK_ERR_ARG (NULL pointers, m < 2, p < 2, k outside 1..p, sweeps outside 1..100),
 *         DK_ERR_UNSUPPORTED (p > DK_PCA_MAX_FEATURES), DK_ERR_WORKSPACE (workspace too small
 *         or misaligned). */
dk_status dk_pca_fit(dk_ctx* ctx, const float* x, int m, int p, int k, int sweeps, void* workspace,
                     size_t workspace_bytes, float* mean, float* scale, float* components, float* eigenvalues,
                     float* off_norm, void* stream);

/* Projection onto the leading k components and min-max scaling (§II-A): y = ((x - mean) /
 * scale) components^T, then out = range_max (y - lo) / (hi - lo) clipped to [0, range_max]
 * (0 where hi == lo). fit_range = 1 (training rows): lo / hi are the per-feature minimum and
 * maximum of y over these rows (written); fit_range = 0 (test rows): lo / hi are read.
 *   x            m x p float32 (device); mean, scale, components from dk_pca_fit
 *   lo, hi       k floats each (device)
 *   out          m x k floats (device, written)
 * Errors: DK_ERR_ARG (NULL pointers, m < 1, p < 1, k outside 1..p, range_max <= 0). */
dk_status dk_pca_transform(dk_ctx* ctx, const float* x, int m, int p, const float* mean, const float* scale,
                           const float* components, int k, int fit_range, float range_max, float* lo, float* hi,
                           float* out, void* stream);

/* Largest feature count of dk_pca_fit_noalloc. */
#define DK_PCA_NOALLOC_MAX_FEATURES 256

/* dk_pca_fit without a caller workspace, for callers that cannot give this library device
 * memory of their own: a program whose device memory is owned and capped by another
 * framework, a plug-in that receives only its input and output pointers, or a loop that must
 * not stall on or fail in an allocation midway. The paper has no counterpart; it is a
 * deployment variant of the §II-A fit above, with the same arguments (minus the workspace)
 * and the same results.
 *   Working memory: a fixed array of about 0.5 MB inside the library (room for
 *   DK_PCA_NOALLOC_MAX_FEATURES features), held by every GPU that loads the library until
 *   the process exits. The call allocates no device memory.
 *   First call on a device: it looks up that array's device address (once per device, with
 *   the context's device made current for the lookup); make this first call before any
 *   stream capture.
 *   Sharing: every call uses the same array, so calls whose work overlaps on the GPU (on
 *   different streams, or from different threads) race and corrupt each other; run them one
 *   after another. Nothing from an earlier call needs clearing: each call writes every part
 *   of the array it reads.
 * Errors: as dk_pca_fit, and DK_ERR_UNSUPPORTED for p > DK_PCA_NOALLOC_MAX_FEATURES;
 *         DK_ERR_CUDA if the array's address cannot be found. */
dk_status dk_pca_fit_noalloc(dk_ctx* ctx, const float* x, int m, int p, int k, int sweeps, float* mean, float* scale,
                             float* components, float* eigenvalues, float* off_norm, void* stream);

/* Largest training list (m_max) of the SVM calls below. */
#define DK_SVM_MAX_SAMPLES 4096

/* One-against-one SVM training on precomputed kernel values (§II-B, Eqs. 1-2: the dual
 * problem min 1/2 sum a_i a_j y_i y_j K_ij - sum a_i, sum a_i y_i = 0, 0 <= a_i <= C;
 * §II-D, Eq. 11: the mixed kernel), for n_jobs independent jobs in one launch, e.g. the
 * folds x C x w grid of a cross-validation.
 *   kq, kc     n x n kernel matrices over the samples (device, float32, row stride ld >= n);
 *              the job uses K(r, c) = w[job] kq[r*ld + c] + (1 - w[job]) kc[r*ld + c]. Either
 *              may be NULL (its term is dropped). Only entries between samples of a job are
 *              read.
 *   w, C       n_jobs floats each (device): mixing weight and box bound per job
 *   idx        n_jobs x m_max int32 (device): job j trains on the samples idx[j*m_max + k],
 *              k < count[j] (indices 0..n-1 into the kernel matrix), in this order; an index
 *              outside 0..n-1 is skipped and makes the next dk_sync_status return DK_ERR_ARG
 *   count      n_jobs int32 (device), each in 0..m_max (larger values act as m_max)
 *   labels     class of every sample, indexed like the kernel matrix (device int32,
 *              0..n_class-1)
 *   tol        stop when the largest KKT violation (max over the upper set minus min over the
 *              lower set of -y_t grad_t) is below tol
 *   max_iter   steps per binary problem at most
 * For class pair p = (c1, c2), c1 < c2, numbered (0,1), (0,2), ..., (1,2), ..., one binary
 * problem on the job's samples of those two classes with y = +1 for c1, solved by
 * sequential minimal optimisation with second-order working-set selection.
 *   coef       n_jobs x P x m_max floats, P = n_class (n_class - 1) / 2 (device, written):
 *              a_k y_k of the sample at position k of the job's list; 0 for samples outside
 *              the pair and for k >= count[j]
 *   bias       n_jobs x P floats (device, written): b of the decision function (Eq. 5)
 *   iters      n_jobs x P int32 (device, written, may be NULL): steps taken, -1 if max_iter
 *              was reached before tol; 0 when a class of the pair is absent from the job
 *              (coef and bias are then 0)
 * Errors: DK_ERR_ARG (NULL ctx / w / C / idx / count / labels / coef / bias, both kq and kc
 *         NULL, n_jobs outside 1..65535, m_max < 2, n < 1, ld < n, tol <= 0, max_iter < 1),
 *         DK_ERR_UNSUPPORTED (n_class outside 2..32, m_max > DK_SVM_MAX_SAMPLES). */
dk_status dk_svm_ovo_train(dk_ctx* ctx, const float* kq, const float* kc, long long ld, int n, int n_jobs,
                           const float* w, const float* C, const int32_t* idx, const int32_t* count,
                           int m_max, const int32_t* labels, int n_class, float tol, int max_iter,
                           float* coef, float* bias, int32_t* iters, void* stream);

/* Decision values and one-against-one votes (§II-B, Eqs. 4-5) for rows of a kernel matrix,
 * per job of dk_svm_ovo_train.
 *   kq, kc, ld, w  as for dk_svm_ovo_train, but n_rows x n_cols (n_cols <= ld): K(r, c) is
 *              read at row r of the classified samples and column c of the training samples
 *              (for test samples: the output of dk_dual_kernel_rows)
 *   rows       n_jobs x r_max int32 (device) row indices 0..n_rows-1 of the samples to
 *              classify, or NULL for rows 0..r_max-1; row_count n_jobs int32 (device) or NULL
 *              for r_max. A row index out of range is not classified and makes the next
 *              dk_sync_status return DK_ERR_ARG, as does a training index outside 0..n_cols-1
 *              (that sample then contributes nothing).
 *   idx, count the training lists of the jobs (device), or NULL for columns 0..m_max-1
 *   coef, bias the outputs of dk_svm_ovo_train for the same jobs and m_max
 *   decision   n_jobs x r_max x P floats (device, written, may be NULL): f_p(x) of Eq. 5
 *   pred       n_jobs x r_max int32 (device, written, may be NULL): the class with the most
 *              votes (pair (c1, c2) votes c1 if f > 0, else c2), the smallest index on ties
 * Entries of rows past row_count[j] are not written.
 * Errors: DK_ERR_ARG (NULL ctx / w / coef / bias, both kq and kc NULL, both decision and
 *         pred NULL, n_jobs outside 1..65535, r_max < 1, m_max < 1, n_rows < 1, n_cols < 1,
 *         ld < n_cols, rows NULL with r_max > n_rows, idx NULL with m_max > n_cols),
 *         DK_ERR_UNSUPPORTED (n_class outside 2..32, m_max > DK_SVM_MAX_SAMPLES). */
dk_status dk_svm_ovo_predict(dk_ctx* ctx, const float* kq, const float* kc, long long ld, int n_rows,
                             int n_cols, int n_jobs, const float* w, const int32_t* rows,
                             const int32_t* row_count, int r_max, const int32_t* idx, const int32_t* count,
                             int m_max, const float* coef, const float* bias, int n_class, float* decision,
                             int32_t* pred, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DUALK_H */
