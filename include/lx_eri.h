/*
 * lx_eri.h -- C ABI of a GB300 (sm_103a) library that evaluates batches of 4-center
 * 2-electron repulsion integrals (ab|cd) over contracted Cartesian Gaussian shells by
 * the matrix form of the McMurchie-Davidson (MD) recurrences (Asadchev & Valeev,
 * "High-performance evaluation of high angular momentum 4-center Gaussian integrals on
 * modern accelerated processors", arXiv:2307.03452).
 *
 * What is computed (paper, Section 2 "Formalism"):
 *   (ab|cd) = sum_{p,q} H_ab^p [p|q] H_cd^q   over all primitive quartets,
 *   [p|q]   = (-1)^{l_q} [p+q]^(0)                                     (Eq. pq)
 *   [r+1_i]^(m) = r_i [r-1_i]^(m+1) + (P_i - Q_i) [r]^(m+1)             (Eq. md1)
 *   [0]^(m) = (-2 rho)^m 2 pi^{5/2} / (zeta_p zeta_q sqrt(zeta_p+zeta_q)) F_m(rho |PQ|^2)
 *   F_m(T)  = int_0^1 y^{2m} exp(-T y^2) dy                             (Eq. boys)
 *   H_ab^p  = sum_{a,b} C^a_{l_a m_a} C^b_{l_b m_b} E_ab^p  (solid) or E_ab^p (Cartesian),
 *   with E from the recursions after Eq. cart2herm-2, evaluated as the two transforms
 *   Eq. ab_to_hermite / Eq. make-abq and Eq. cd_to_hermite / Eq. make-abcd.
 *
 * Conventions (the paper leaves them open):
 *   - Cartesian components of a shell l in the order: for i = 0..l, j = 0..i:
 *     (l-i, i-j, j).  Every component carries the normaliser of x^l exp(-zeta r^2).
 *   - Raw contraction coefficients are normalised inside the library: c_i times the
 *     primitive normaliser, rescaled so that the contracted x^l function has unit norm.
 *   - Real solid harmonics are unit-normalised, ordered m = -l..l (Schlegel & Frisch).
 *   - A quartet's output block is row-major over (a, b, c, d) components, written at
 *     out + out_offset (in doubles).
 *   - No screening is done (the paper's Section 3: the caller screens).
 *
 * Threading: every entry point is thread-safe; the first call on a device uploads
 * constant tables to that device (synchronously), so make it before any stream capture.
 */
#ifndef LX_ERI_H
#define LX_ERI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LX_LMAX 7  /* largest shell angular momentum (k shells) */
#define LX_KMAX 16 /* largest contraction degree of one shell */

/* One shell: angular momentum l (0..LX_LMAX), nprim primitives whose exponents and raw
   contraction coefficients start at exps[prim_offset] / coefs[prim_offset], center in bohr. */
typedef struct {
    int32_t l;
    int32_t nprim;
    int32_t prim_offset;
    int32_t reserved; /* must be 0 */
    double center[3];
} lx_shell;

/* One shell quartet (ab|cd): shell indices s[0..3] = a, b, c, d and the offset (in doubles)
   of its output block in the caller's output buffer. */
typedef struct {
    int32_t s[4];
    int64_t out_offset;
} lx_quartet;

/* flags */
#define LX_CART 0x0        /* Cartesian output, ncart(l) = (l+1)(l+2)/2 per shell */
#define LX_SOLID 0x1       /* real solid-harmonic output, 2l+1 per shell */
#define LX_PATH_FP64 0x0   /* every step in FP64 */
#define LX_PATH_SPLIT 0x2  /* the two Hermite transforms as Ozaki-style BF16 slice products on the
                              tensor cores (FP32 accumulation, integer recombination); Boys,
                              [r]^(m), E and H stay FP64.  Operands carry 8 bits per digit kept
                              (48 with the default 6 digits); the absolute error grows with the
                              magnitude of a quartet's intermediates */
#define LX_SPLIT_DIGITS(n) (((n) & 7) << 4) /* with LX_PATH_SPLIT: BF16 digits kept per operand
                              value, n = 4, 5 or 6 (the default, also given by 0); the transforms
                              keep the n(n+1)/2 digit products with s + t < n, and each digit
                              fewer multiplies the error by about 2^8 */
#define LX_SPLIT_DIGITS_MASK 0x70
#define LX_PATH_ROUTED 0x4 /* per quartet: the routing network set by lx_router_set predicts
                              log10 of the split path's error on the quartet (its output 1); the
                              quartet takes the split path with the fewest digits (4, 5, 6) whose
                              threshold lies above that prediction, else LX_PATH_FP64.  Quartets
                              whose two transforms need fewer than LX_ROUTE_SPLIT_MIN_FLOP FLOPs
                              (too small for the split path to be faster) take LX_PATH_FP64.
                              lx_eri_batch then waits for the stream once, to read the predictions
                              back.  Not with LX_PATH_SPLIT; not for lx_eri_graph_create,
                              lx_eri_autotune or lx_eri_batch_static */
#define LX_ROUTE_SPLIT_MIN_FLOP 1.0e6 /* 2 N_ab (K_bra N_p)(K_ket N_q) + 2 N_ab (K_ket N_q) N_cd */
#define LX_TIME_STAGES 0x200 /* record CUDA events around each stage (see lx_eri_stage_times) */

/* stages timed with LX_TIME_STAGES */
#define LX_STAGE_NORM 0   /* contraction normalisation */
#define LX_STAGE_PAIR 1   /* pair scalars and H matrices */
#define LX_STAGE_BOYS_R 2 /* Boys function and [r]^(0) */
#define LX_STAGE_GEMM1 3  /* [ab|q] = H_ab [p|q] */
#define LX_STAGE_GEMM2 4  /* (ab|cd) = [ab|q] H_cd^T */
#define LX_STAGE_SPLIT 5  /* LX_PATH_SPLIT: FP64 operands -> BF16 digit planes */
#define LX_STAGE_DIGEST 6 /* lx_eri_jk: blocks digested into J and K */
#define LX_NSTAGE 7

/* error codes (0 = success) */
#define LX_OK 0
#define LX_ERR_NULL (-1)          /* a required pointer is NULL */
#define LX_ERR_SHELL (-2)         /* l outside 0..LX_LMAX, nprim outside 1..LX_KMAX, reserved != 0,
                                     primitive range outside the arrays, or non-finite center */
#define LX_ERR_PRIMITIVE (-3)     /* exponent not finite and > 0, or coefficient not finite */
#define LX_ERR_QUARTET (-4)       /* shell index out of range or negative out_offset */
#define LX_ERR_FLAGS (-5)         /* unknown flag bits */
#define LX_ERR_WORKSPACE (-6)     /* workspace NULL or smaller than lx_eri_workspace_min */
#define LX_ERR_CUDA (-7)          /* a CUDA runtime call failed (see lx_last_cuda_error) */
#define LX_ERR_ARCH (-8)          /* current device is not compute capability 10.3 */
#define LX_ERR_DEVICE_STATUS (-9) /* a kernel reported a bad index or an exhausted wait */
#define LX_ERR_SIZE (-10)         /* a size argument is negative or too large */
#define LX_ERR_STATIC_SCRATCH (-11) /* lx_eri_batch_static: the batch needs more scratch than
                                       LX_STATIC_SCRATCH_BYTES even one quartet at a time */
#define LX_ERR_NO_ROUTER (-12)    /* LX_PATH_ROUTED on a device without lx_router_set */
#define LX_ERR_PAIR_CLASS (-13)   /* lx_eri_pairs*: the bra (or ket) pairs differ in (l, l') */

/*
 * Number of doubles the output buffer needs: max over quartets of out_offset + block size.
 * Host pointers.  Returns a negative error code on invalid input.
 */
int64_t lx_eri_out_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets, int64_t nquartet,
                        int32_t flags);

/*
 * Device workspace (bytes) to evaluate the whole batch in one pass.  A smaller workspace
 * (at least lx_eri_workspace_min) also works: the batch is then processed in chunks.
 */
int64_t lx_eri_workspace_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                              int64_t nquartet, int32_t flags);

/* Smallest workspace (bytes) with which lx_eri_batch accepts this batch (one quartet at a time). */
int64_t lx_eri_workspace_min(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                             int64_t nquartet, int32_t flags);

/*
 * Evaluate (ab|cd) for every quartet.
 *   shells[nshell], exps[nprim_total], coefs[nprim_total], quartets[nquartet]: HOST memory,
 *     read during the call only.
 *   out: DEVICE memory (current device), caller-owned, at least lx_eri_out_size doubles;
 *     only the quartets' blocks are written.
 *   workspace: DEVICE memory, caller-owned, workspace_bytes long, 256-byte aligned; it
 *     holds the per-call descriptors, the H matrices, the [r]^(0) vectors and the
 *     intermediate [ab|q] blocks.  It must not be reused until the stream has passed the work.
 *   cuda_stream: a cudaStream_t of the current device (NULL = legacy default stream).
 * The call validates every input on the host, plans the batch, copies the planned
 * descriptors into page-locked staging memory owned by the library (a few buffers per
 * device, reused once their uploads have completed), enqueues the uploads and the kernels
 * and returns without waiting for them.  Errors found on the device are reported by
 * lx_eri_sync_status.  A stream in capture mode is refused (LX_ERR_CUDA): capture a batch
 * with lx_eri_graph_create.
 */
int lx_eri_batch(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                 int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                 void* workspace, size_t workspace_bytes, void* cuda_stream);

/*
 * Bra-list x ket-list form (Section 3, the library interface): (ab|cd) for every bra pair i
 * and every ket pair j.
 *   bra_pairs[2 nbra], ket_pairs[2 nket]: HOST int32 shell indices (a, b) and (c, d).  Every
 *     bra pair has the same (l_a, l_b) and every ket pair the same (l_c, l_d)
 *     (LX_ERR_PAIR_CLASS otherwise); contraction degrees may differ.
 *   out: DEVICE, dense [nbra][nket][n_ab][n_cd] (n(l) functions per shell as for
 *     lx_eri_batch), lx_eri_pairs_out_size = nbra nket n_ab n_cd doubles.
 * Otherwise as lx_eri_batch, which it calls with the quartets (i | j) in bra-major order:
 * within one chunk of the workspace every pair's H matrix (and, on the split path, its
 * column scales and BF16 digit planes) is built once and shared by all the chunk's quartets
 * that contain the pair.  nbra nket <= LX_PAIRS_MAX_QUARTETS (LX_ERR_SIZE otherwise).
 */
#define LX_PAIRS_MAX_QUARTETS (1ll << 28)
int64_t lx_eri_pairs_out_size(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                              const int32_t* ket_pairs, int64_t nket, int32_t flags);
int64_t lx_eri_pairs_workspace_size(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                                    const int32_t* ket_pairs, int64_t nket, int32_t flags);
int64_t lx_eri_pairs_workspace_min(const lx_shell* shells, int32_t nshell, const int32_t* bra_pairs, int64_t nbra,
                                   const int32_t* ket_pairs, int64_t nket, int32_t flags);
int lx_eri_pairs(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
                 const int32_t* bra_pairs, int64_t nbra, const int32_t* ket_pairs, int64_t nket, int32_t flags,
                 double* out, void* workspace, size_t workspace_bytes, void* cuda_stream);

/*
 * Coulomb and exchange digestion (Section 3: Fock matrix elements formed from the integral
 * batches directly).  Basis functions are numbered shell by shell in the order of shells[]:
 * shell s owns functions bf(s) .. bf(s) + n(l_s) - 1, bf(s) = sum over s' < s of n(l_s'),
 * with n(l) = 2l+1 (LX_SOLID) or (l+1)(l+2)/2; lx_nbf returns the total nbf.  For every
 * listed quartet (ab|cd), mu in a, nu in b, lam in c, sig in d:
 *     J[mu][nu]  += sum_{lam, sig} (mu nu|lam sig) D[lam][sig]
 *     K[mu][lam] += sum_{nu, sig}  (mu nu|lam sig) D[nu][sig]
 * Each quartet counts once as listed (the caller lists the permutational images it wants
 * and folds their degeneracy into D or the list).
 *   D: DEVICE, nbf x nbf row-major, read only.  J, K: DEVICE, nbf x nbf row-major, added to
 *     (atomically: the summation order, and so the last bits, vary from run to run); either
 *     may be NULL to skip it, not both.
 *   quartets[].out_offset is not used (it must still be >= 0).
 *   workspace: as lx_eri_batch, sized by lx_eri_jk_workspace_size / _min.  On the FP64
 *     path J and K are contracted straight from [ab|q] (no second transform, no block
 *     stored); on the split path each quartet's block is written to the workspace by the
 *     second transform and streamed once by the digestion kernel.  Nothing is written to a
 *     caller output.
 * Flags, paths (LX_PATH_SPLIT, LX_PATH_ROUTED), staging and stream semantics as
 * lx_eri_batch; LX_TIME_STAGES times the digestion as LX_STAGE_DIGEST.  nbf <= 2^31 - 1.
 */
int64_t lx_nbf(const lx_shell* shells, int32_t nshell, int32_t flags);
int64_t lx_eri_jk_workspace_size(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                                 int64_t nquartet, int32_t flags);
int64_t lx_eri_jk_workspace_min(const lx_shell* shells, int32_t nshell, const lx_quartet* quartets,
                                int64_t nquartet, int32_t flags);
int lx_eri_jk(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs, int32_t nprim_total,
              const lx_quartet* quartets, int64_t nquartet, int32_t flags, const double* D, double* J, double* K,
              void* workspace, size_t workspace_bytes, void* cuda_stream);

/*
 * lx_eri_batch without a workspace argument, for callers that cannot allocate device memory
 * (for example a plugin whose host program owns every device allocation through its own
 * pool, or a process in which cudaMalloc is not permitted).  There is no counterpart in the
 * paper; it exists only for such callers.
 *   Same inputs, output and stream semantics as lx_eri_batch.  The scratch is a fixed array
 *   of LX_STATIC_SCRATCH_BYTES inside the library's device image: every GPU that loads the
 *   library holds it until the process exits.  The call allocates no device memory of its
 *   own; the first call of any entry point on a device (this one included) uploads the
 *   library's constant tables there once (the solid-fold row lists and the split path's
 *   [p+q] index table, about 45 MB, held until exit), so a caller that must not allocate
 *   makes that first call where allocation is still allowed.  The first call on a device
 *   also looks up the array's device address (cudaGetSymbolAddress, with that device
 *   current); make that first call before any stream capture.
 *   A stream in capture mode is refused (LX_ERR_CUDA): the call uploads its descriptors from
 *   host memory that it releases on return.  LX_PATH_ROUTED and LX_TIME_STAGES are refused
 *   (LX_ERR_FLAGS): routing needs scratch beyond the array, and stage timing creates CUDA
 *   events.
 *   A batch whose smallest workspace (lx_eri_workspace_min) exceeds LX_STATIC_SCRATCH_BYTES
 *   is rejected with LX_ERR_STATIC_SCRATCH; larger batches that fit one quartet at a time are
 *   processed in chunks.
 *   All calls on a device share the one array: calls that overlap on the GPU (for example on
 *   two streams at once) race and give wrong results; serialise them on one stream.  The
 *   array keeps the last call's contents; the pipeline never reads scratch it has not
 *   written in the same call.
 */
#define LX_STATIC_SCRATCH_BYTES (64ull << 20)
int lx_eri_batch_static(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                        int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags,
                        double* out, void* cuda_stream);

/*
 * Capture the whole evaluation of a batch into a CUDA graph bound to `out` and `workspace`
 * (same arguments and meaning as lx_eri_batch, LX_TIME_STAGES not allowed): every stage of
 * every chunk, over quartets of any mix of classes and contraction degrees, then replays with
 * one lx_eri_graph_launch.  The descriptors are copied into pinned host memory owned by the
 * handle, so the host arrays may be freed after the call.  *handle receives the graph.
 */
int lx_eri_graph_create(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                        int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags,
                        double* out, void* workspace, size_t workspace_bytes, void** handle);
/* Enqueue one replay of a captured batch on cuda_stream (asynchronous). */
int lx_eri_graph_launch(void* handle, void* cuda_stream);
/* Release a captured batch (after its last replay has completed). */
int lx_eri_graph_destroy(void* handle);

/*
 * Autotune the tile shape of the two FP64 GEMM stages per (l_a, l_b, l_c, l_d, K_bra, K_ket,
 * output kind): for each of the `max_keys` costliest keys of the batch, up to `samples` of its
 * quartets are evaluated with every tile shape (32x64, 64x32, 32x32, 64x64) and the fastest,
 * timed with CUDA events on cuda_stream, is recorded in the library's tuning table, which the
 * planner consults for every later call.  out (DEVICE, out_doubles long) and workspace are
 * scratch.  Synchronises cuda_stream.  The split path has a single tile shape: no-op.
 */
int lx_eri_autotune(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                    int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags, double* out,
                    int64_t out_doubles, void* workspace, size_t workspace_bytes, int32_t max_keys, int32_t samples,
                    void* cuda_stream);
/* Tuning table rows (9 int32 each: l_a, l_b, l_c, l_d, K_bra, K_ket, solid, shape of GEMM1,
   shape of GEMM2): export writes min(count, cap) rows and returns the count; import adds or
   replaces rows (LX_ERR_SIZE on an invalid row, nothing imported); clear empties the table. */
int64_t lx_tune_export(int32_t* rows, int64_t cap);
int lx_tune_import(const int32_t* rows, int64_t n);
int lx_tune_clear(void);

/*
 * Wait for cuda_stream, then read and clear the device status word of the current device.
 * Returns LX_OK, LX_ERR_DEVICE_STATUS if a kernel flagged an error since the last call,
 * or LX_ERR_CUDA if the stream reported a CUDA error.
 */
int lx_eri_sync_status(void* cuda_stream);

/*
 * Milliseconds spent in each stage (ms[LX_STAGE_*], nstage <= LX_NSTAGE) and the number of
 * kernel launches per stage (launches[], may be NULL), summed over every lx_eri_batch call
 * made with LX_TIME_STAGES on cuda_stream since the previous call of this function; the
 * accumulators are then cleared.  Waits for cuda_stream.  The events are recorded on the
 * stream the kernels run on, so each figure is the stage's device time.
 */
int lx_eri_stage_times(double* ms, int64_t* launches, int32_t nstage, void* cuda_stream);

/*
 * Failure-detection self-test: enqueue on cuda_stream one wait of `tries` attempts
 * (tries <= 2^24, the limit of the library's own waits) on a barrier that nothing
 * arrives on -- the path every bounded wait of the library takes when its partner never
 * comes.  The kernel sets the device status word's timeout bit and returns; the next
 * lx_eri_sync_status reports LX_ERR_DEVICE_STATUS (and clears the word), and the device
 * stays usable.  Returns LX_OK once enqueued.
 */
int lx_selftest_timeout(uint64_t tries, void* cuda_stream);

/* Human-readable text of an error code (static storage). */
const char* lx_strerror(int code);

/* Text of the last CUDA error seen by this thread (static thread-local storage). */
const char* lx_last_cuda_error(void);

/* ---------------------------------------------------------------- stage entry points
 * The same device routines the batch path uses, exposed one stage at a time so that each
 * stage can be checked on its own.  All array arguments are DEVICE pointers. */

/*
 * Boys function, Eq. boys: F[i*(mmax+1) + m] = F_m(T[i]) for m = 0..mmax, i < n.
 * mmax <= 4*LX_LMAX; T[i] >= 0 and finite (a negative or non-finite T sets the device
 * status word and yields NaN).  Tabulated Taylor expansion plus downward recursion for
 * T < 36, erf-free asymptotic F_0 plus upward recursion above.
 */
int lx_boys(int32_t mmax, const double* T, int64_t n, double* F, void* cuda_stream);

/*
 * Auxiliary Hermite integrals [r]^(0), |r| <= L, by Eq. md1 in place with descending m.
 * Item i: params[5i..5i+4] = (rho, PQx, PQy, PQz, pref) with pref the prefactor
 * 2 pi^{5/2}/(zeta_p zeta_q sqrt(zeta_p+zeta_q)); output R[i*pyr(L) + idx(t,u,v)] with the
 * pyramidal index idx(t,u,v) = n(n+1)(n+2)/6 + i'(i'+1)/2 + v, n = t+u+v, i' = u+v,
 * pyr(L) = (L+1)(L+2)(L+3)/6.  L <= 4*LX_LMAX.
 */
int lx_hermite_R(int32_t L, const double* params, int64_t n, double* R, void* cuda_stream);

/*
 * Hermite-to-Cartesian/solid matrices H (Section 2, definition of H) of shell pairs.
 * pairs[2k], pairs[2k+1]: shell indices (a, b) of pair k (HOST memory, like shells, exps,
 * coefs).  Output H (DEVICE) for pair k starts at H + k*stride with
 * stride = max over pairs of nfun(l_a) nfun(l_b) K_a K_b pyr(l_a+l_b), laid out as
 * [a b][kp * pyr(l_a+l_b) + idx(p)] with kp = i_a K_b + i_b the primitive pair; each row
 * carries exp(-mu |AB|^2) and the normalised coefficients of both primitives.  flags:
 * LX_SOLID selects solid output; bit 0x100 multiplies column p by (-1)^{|p|} (ket side).
 */
int lx_hermite_H(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                 int32_t nprim_total, const int32_t* pairs, int32_t npair, int32_t flags, double* H,
                 int64_t stride, void* cuda_stream);

/*
 * C = A B^T through the split path's kernels (the same splitting and tensor-core GEMM that
 * LX_PATH_SPLIT uses for Eq. make-abq / Eq. make-abcd): A is M x K, B is N x K, both FP64
 * row-major in DEVICE memory with row strides lda, ldb; C is M x N FP64 row-major, stride ldc.
 * Each row of A and of B is scaled by its own power of two and split into BF16 digits of
 * 8 bits, of which `digits` (4, 5 or 6) are kept; the digit products with s + t < digits
 * are summed.  Scratch for the digit planes is taken from the stream-ordered allocator.
 * M, N, K >= 1, K <= 1 << 20.
 */
int lx_split_gemm(int32_t M, int32_t N, int32_t K, const double* A, int32_t lda, const double* B, int32_t ldb,
                  double* C, int32_t ldc, int32_t digits, void* cuda_stream);

/* ---------------------------------------------------------------- learned router
 * A small MLP predicts, per quartet from shell descriptors, log10 of its largest |integral|
 * (output 0) and log10 of the split path's absolute error on it with 6 digits (output 1),
 * which follows the magnitude of the quartet's intermediates rather than of its result when
 * the Hermite sums cancel.  LX_PATH_ROUTED sends each quartet to the split path with as few
 * digits as that prediction allows, or to LX_PATH_FP64.  The paper has no such part.
 * Network: LX_MLP_NIN inputs -> 64 -> 64 -> LX_MLP_NOUT, ReLU, parameters packed as
 * W1[64][20], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]; the forward pass uses FP16
 * weights. */
#define LX_MLP_NIN 20
#define LX_MLP_WIDTH 64
#define LX_MLP_NOUT 2
#define LX_MLP_NPARAM (LX_MLP_WIDTH * LX_MLP_NIN + LX_MLP_WIDTH + LX_MLP_WIDTH * LX_MLP_WIDTH + LX_MLP_WIDTH + \
                       LX_MLP_NOUT * LX_MLP_WIDTH + LX_MLP_NOUT)
#define LX_ROUTE_NTIER 3 /* split tiers of LX_PATH_ROUTED: 4, 5 and 6 digits */

/*
 * Router features of each quartet: feat[q * LX_MLP_NIN + k] (DEVICE, float).  Descriptors are
 * HOST arrays as for lx_eri_batch (coefficients are not needed).  Features: l / 6 of each
 * shell; ln of the smallest and largest exponent of each shell / 4; |AB|, |CD| / 10; the
 * distance of the most diffuse product centers / 30; mu |AB|^2 and nu |CD|^2 of the most
 * diffuse primitives / 20; ln(1 + rho |PQ|^2) / 3; ln(Ka Kb Kc Kd) / 6; log10 of an
 * (ss|ss)-type magnitude estimate / 10.  Scratch comes from the stream-ordered allocator.
 */
int lx_route_features(const lx_shell* shells, int32_t nshell, const double* exps, int32_t nprim_total,
                      const lx_quartet* quartets, int64_t nquartet, float* feat, void* cuda_stream);

/*
 * The routing network of LX_PATH_ROUTED on the current device: params_f16 holds the
 * LX_MLP_NPARAM FP16 parameters (HOST memory, layout as above); tau[LX_ROUTE_NTIER] (HOST)
 * the thresholds on output 1 for the split tiers of 4, 5 and 6 digits: a quartet takes the
 * first tier, in that order, whose threshold lies above its prediction, and the FP64 path if
 * none does (a tier is disabled by a threshold of -1e30).  The parameters are copied
 * (synchronously); a later call replaces them.  Thresholds must be finite.
 */
int lx_router_set(const void* params_f16, const float* tau);

/* Inference: out[i * LX_MLP_NOUT + o] = output o of MLP(feat[i]) with FP16 parameters
 * params_f16 (DEVICE, LX_MLP_NPARAM halves). */
int lx_mlp_forward(const void* params_f16, const float* feat, int64_t n, float* out, void* cuda_stream);

/*
 * Training gradient: loss[0] = mean over i < n of sum_o (MLP(feat[i])_o - target[i*LX_MLP_NOUT+o])^2,
 * evaluated with the FP16-rounded params, and grad = its gradient with respect to params
 * (straight through the rounding).  All DEVICE float arrays; grad and loss are overwritten.
 */
int lx_mlp_grad(const float* params, const float* feat, const float* target, int64_t n, float* grad, float* loss,
                void* cuda_stream);

/*
 * One Adam step (step counts from 1) on params with moments m, v (DEVICE, LX_MLP_NPARAM floats
 * each) from grad, which is then cleared; params_f16 receives the rounded parameters.
 */
int lx_mlp_adam(float* params, float* m, float* v, float* grad, void* params_f16, int32_t step, float lr,
                float beta1, float beta2, float eps, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LX_ERI_H */
