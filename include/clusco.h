/*
 * clusco.h -- C-ABI of libclusco: all-versus-all cRMSD on one B300 (sm_103a).
 *
 * The operation (ClusCo, section "Algorithms", eq. 1 and eq. 2): for models A
 * and B of L matched atoms,
 *     cRMSD = sqrt(R_A^2 + R_B^2 - 2 (sqrt(l1) + sqrt(l2) + S sqrt(l3)))
 * where R_A, R_B are the radii of gyration, l1 >= l2 >= l3 the eigenvalues of
 * M^T M for the 3x3 covariance M = (1/L) sum_i a_i b_i^T of the centred
 * coordinates, found as roots of a cubic, and S = sign(det M). This equals the
 * RMS deviation after the optimal superposition (eq. 1) without building the
 * rotation. The all-versus-all matrix has N(N-1)/2 entries (section
 * "Background"); scoring against a reference model is the second mode the
 * paper names (section "Results and Discussion", first paragraph).
 *
 * Conventions shared by every call:
 *  - Pointers named coords, ref, out, grad_out, grad_coords and crmsd are DEVICE pointers owned by
 *    the caller; the library never frees or keeps them. coords is
 *    float[N][L][3] (row-major, atom-major, xyz innermost), 4-byte aligned.
 *  - Condensed output: out[idx(a,b)] for a < b with
 *    idx(a,b) = a*N - a*(a+1)/2 + (b - a - 1)   (int64 arithmetic).
 *  - workspace: optional device scratch of at least
 *    clusco_workspace_bytes(op, N, L, form) bytes, 256-byte aligned. If it is
 *    NULL the call allocates stream-ordered scratch (cudaMallocAsync) and
 *    frees it on the same stream.
 *  - stream: a cudaStream_t (NULL = legacy default stream). Every call only
 *    enqueues work and returns; argument errors return at once and enqueue
 *    nothing.
 *  - Device-detected conditions (non-finite input, a bounded wait that gave
 *    up) set a device status word; clusco_sync_status() synchronises the
 *    stream, returns that status and clears it. A model with a non-finite
 *    coordinate yields NaN for every pair it is in. No call traps the GPU.
 *  - Return values are clusco_status codes; clusco_last_error() gives a
 *    thread-local message for the last non-OK return.
 */
#ifndef CLUSCO_H
#define CLUSCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CLUSCO_OK = 0,
    CLUSCO_EINVAL = 1,      /* bad argument: sizes, null or unaligned pointer, range */
    CLUSCO_ENOMEM = 2,      /* scratch allocation failed / workspace too small */
    CLUSCO_ECUDA = 3,       /* a CUDA runtime call failed (message has the name) */
    CLUSCO_ETIMEOUT = 4,    /* a bounded device wait gave up (device status) */
    CLUSCO_EOVERFLOW = 5,   /* N*L*3 or the condensed index would overflow int64 */
    CLUSCO_ENONFINITE = 6,  /* an input coordinate was NaN or Inf (device status) */
    CLUSCO_EUNSUPPORTED = 7 /* form not available for these sizes / this device */
} clusco_status;

/* Precision forms of the covariance contraction (the epilogue is fixed per form):
 *  FP32_SIMT   -- plain form: FP32 CUDA-core GEMM, FP64 cubic (Viete) epilogue.
 *  TF32        -- tcgen05 kind::tf32 on TF32-rounded centred coordinates.
 *  BF16X3      -- tcgen05 bf16, classic split x = hi + lo, hi*hi + hi*lo + lo*hi
 *                 in one FP32 accumulator.
 *  BF16_EXACT2 -- tcgen05 bf16 on 16-bit fixed point coordinates split in two
 *                 8-bit digits; all four digit products kept in separate FP32
 *                 accumulators, exact for L <= 1024; FP32 epilogue with FP64
 *                 refinement of the pairs whose FP32 error bound is too large.
 *  FP8_EXACT   -- tcgen05 kind::f8f6f4 on 0/1 operands (exact integer counts);
 *                 the tensor-core form of the contact map overlap only.
 *  INT_SIMT    -- exact-integer CUDA-core form: 24-bit fixed point per model and
 *                 axis (step max|x| / (2^23 - 1)), every product a 32 x 32 -> 64-bit
 *                 integer multiply-add into int64 (exact for L <= 2^17); FP32 epilogue
 *                 with FP64 refinement of every pair whose FP32 error bound exceeds
 *                 2e-5 A. All-pairs calls (dense, panel, threshold) only; no rotations,
 *                 no fused step, no dRMSD / CMO (CLUSCO_EUNSUPPORTED). */
typedef enum {
    CLUSCO_FORM_FP32_SIMT = 0,
    CLUSCO_FORM_TF32 = 1,
    CLUSCO_FORM_BF16X3 = 2,
    CLUSCO_FORM_BF16_EXACT2 = 3,
    CLUSCO_FORM_FP8_EXACT = 4,
    CLUSCO_FORM_INT_SIMT = 5
} clusco_form;

typedef enum {
    CLUSCO_OP_ALLPAIRS = 0,
    CLUSCO_OP_VS_REF = 1,
    CLUSCO_OP_BACKWARD = 2,
    CLUSCO_OP_BACKWARD_ROT = 3,
    CLUSCO_OP_ALLPAIRS_ROT = 4,
    CLUSCO_OP_DRMSD = 5,
    CLUSCO_OP_CMO = 6,
    CLUSCO_OP_STEP_ROT = 7,
    CLUSCO_OP_STEP = 8
} clusco_op;

/* Library version (major*10000 + minor*100 + patch). */
int clusco_version(void);

/* Bytes of device workspace op needs for (N, L, form); 0 on invalid sizes. */
size_t clusco_workspace_bytes(int op, int64_t N, int64_t L, int form);

/* All-versus-all condensed cRMSD matrix (eq. 2 for every pair a < b).
 * coords: float[N][L][3] device; out: float[N(N-1)/2] device, overwritten.
 * N >= 2, L >= 1. Forms as above; FP32 output. */
int clusco_crmsd_allpairs(const float *coords, int64_t N, int64_t L, float *out, int form,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Row panel of the condensed matrix: rows a in [row_begin, row_end), all b > a.
 * out_panel receives exactly those entries, in condensed order, starting at
 * idx(row_begin, row_begin + 1). Panels are idempotent, so a long run can be
 * resumed at any panel boundary. 0 <= row_begin < row_end <= N - 1. */
int clusco_crmsd_allpairs_panel(const float *coords, int64_t N, int64_t L, int64_t row_begin,
                                int64_t row_end, float *out_panel, int form, void *workspace,
                                size_t workspace_bytes, void *stream);

/* Pairs within a cRMSD threshold (section "Selecting of pairs of models within a given cRMSD
 * threshold": the pairs with cRMSD below a cutoff, there 3.2 A, instead of the whole matrix).
 * Appends every pair a < b whose cRMSD, exactly as clusco_crmsd_allpairs computes it in the
 * same form, is < tau (strictly; NaN never qualifies): list[k] = its condensed index
 * idx(a, b) = a N - a (a + 1) / 2 + (b - a - 1) (int64), vals[k] = its cRMSD (FP32), for
 * k < min(*count, cap), in no particular order. *count (device, uint64) is reset by the call
 * and ends as the number of qualifying pairs, also when that exceeds cap: entries past cap are
 * dropped, and the caller can call again with cap >= *count. No dense output is written.
 * list (8-byte aligned) and vals may be NULL when cap = 0; tau may be +inf (every finite pair).
 * Workspace: that of CLUSCO_OP_ALLPAIRS. */
int clusco_crmsd_allpairs_below(const float *coords, int64_t N, int64_t L, float tau, int64_t *list,
                                float *vals, int64_t cap, uint64_t *count, int form, void *workspace,
                                size_t workspace_bytes, void *stream);

/* All-versus-all dRMSD (section "Algorithms", eq. 5): out[idx(a,b)] for a < b, condensed as
 * above, the RMS difference of the two models' intra-model distances over the L (L - 1) / 2
 * atom pairs i < j. No superposition; a mirror image scores 0. coords: float[N][L][3] device.
 * Forms:
 *  CLUSCO_FORM_BF16_EXACT2 -- every distance rounded to 16-bit fixed point with one scale q
 *    and one offset for the ensemble (q = largest distance / 65278); the Gram matrix of the
 *    rounded distances on tcgen05 as four exact BF16 digit classes, drained to int64 every
 *    1024 terms, so the result is the exact dRMSD of the rounded distances: |error| <= q plus
 *    FP32 rounding of the distances (about q / 4 for near-identical models).
 *  CLUSCO_FORM_FP32_SIMT -- FP32 distances, squared differences summed directly on CUDA cores.
 * Other forms return CLUSCO_EUNSUPPORTED. 2 <= N <= 2^24, 2 <= L <= 4096. A model with a
 * non-finite coordinate gives NaN for its pairs (and sets CLUSCO_ENONFINITE in the device status).
 * Workspace: clusco_workspace_bytes(CLUSCO_OP_DRMSD, N, L, form), about 2 N L^2 bytes
 * (the rounded or FP32 distances of every model). */
int clusco_drmsd_allpairs(const float *coords, int64_t N, int64_t L, float *out, int form, void *workspace,
                          size_t workspace_bytes, void *stream);

/* All-versus-all contact map overlap (section "Algorithms", eq. 6 and eq. 7): out[idx(a,b)] for
 * a < b, condensed as above, S = 100 * 2 n(A and B) / (n(A) + n(B)) in percent, with contact maps
 * C_ij = [ |x_i - x_j| < cutoff ] over the atom pairs i < j (the test taken in FP32 as
 * fma(dx, dx, fma(dy, dy, dz * dz)) < cutoff^2) and n(.) their contact counts; S = 0 where
 * neither model has a contact, NaN for a model with a non-finite coordinate (which also sets
 * CLUSCO_ENONFINITE in the device status). The counts are exact integers in both forms, so
 * the score is the FP32 rounding of the exact ratio:
 *  CLUSCO_FORM_FP8_EXACT -- maps as E4M3 0/1 bytes, n(A and B) by tcgen05 kind::f8f6f4 (needs sm_103);
 *  CLUSCO_FORM_FP32_SIMT -- the plain CUDA-core form: maps packed to bits, AND + population count.
 * Other forms return CLUSCO_EUNSUPPORTED. cutoff > 0 and finite (A; 8 A is the customary C-alpha
 * value, the paper gives none). 2 <= N <= 2^24, 2 <= L <= 4096.
 * Workspace: clusco_workspace_bytes(CLUSCO_OP_CMO, N, L, form), about N L^2 / 2 bytes. */
int clusco_cmo_allpairs(const float *coords, int64_t N, int64_t L, float cutoff, float *out, int form,
                        void *workspace, size_t workspace_bytes, void *stream);

/* GDT_TS, TM-score and MaxSub of every model against a reference (section "Algorithms", eq. 3
 * and eq. 4; MaxSub is the TM-score with d0 = 3.5 A): out[3 a + 0] = GDT_TS as a fraction
 * (max C_1 + max C_2 + max C_4 + max C_8) / (4 L), C_x = number of atoms with d < x A;
 * out[3 a + 1] = TM-score with d0 = max(1.24 (L - 15)^(1/3) - 1.8, 0.5) A; out[3 a + 2] = MaxSub.
 * Each is the maximum over the superpositions of one search: seeds are the contiguous fragments
 * of 4, L/4, L/2 and L atoms (lengths below 3 dropped, repeats once); the model is superimposed on
 * the reference by the optimal proper rotation and translation of the seed's atoms, scored, then
 * superimposed again on the atoms within 3.5 A until their number has not changed in four
 * iterations (four refinements in a row select as many atoms as the one before), fewer than 3
 * remain, or 20 refinements were made (a refinement that selects exactly the atoms it was fitted
 * on ends the search too: every later one is the same). Distances and the integer decisions in FP64; TM terms summed in
 * FP32. coords float[N][L][3], ref float[L][3], out float[N][3], all device. 3 <= L <= 1024,
 * N >= 1. A model (or reference) with a non-finite coordinate gives NaN scores and sets
 * CLUSCO_ENONFINITE in the device status. No workspace. */
int clusco_gdt_tm_vs_ref(const float *coords, int64_t N, int64_t L, const float *ref, float *out, void *stream);

/* One-versus-reference: out[a] = cRMSD(model a, ref) for a in [0, N).
 * ref: float[L][3] device; out: float[N] device. Exact-integer covariance on
 * 24-bit fixed point coordinates, FP64 epilogue. N >= 1, L >= 1. */
int clusco_crmsd_vs_ref(const float *coords, int64_t N, int64_t L, const float *ref, float *out,
                        void *workspace, size_t workspace_bytes, void *stream);

/* Largest reference (atoms) accepted by clusco_crmsd_vs_ref_noalloc. */
#define CLUSCO_NOALLOC_MAX_L 16384

/* One-versus-reference that allocates no device memory, for callers that cannot call
 * cudaMalloc: code whose device memory belongs to another allocator or pool (a serving
 * process or framework that reserved the GPU's memory up front), and latency-critical
 * callers for whom cudaMalloc's possible device-wide synchronisation and variable latency
 * are not acceptable. Same arguments, result and tolerance as clusco_crmsd_vs_ref, minus
 * the workspace: the quantised reference lives in a fixed static device array of about
 * 192 KB (references of up to CLUSCO_NOALLOC_MAX_L atoms) that every GPU loading the
 * library keeps until the process exits. L above that maximum returns CLUSCO_EINVAL.
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, host-side once the module is loaded, so the address is right
 * after a cudaDeviceReset too); the first call on a device loads the module, so make it
 * before any stream capture.
 * Every call shares the one array and overwrites all of it that it reads, so nothing
 * needs clearing between calls, but two calls whose kernels can overlap on the GPU
 * (unordered streams) race on it and may return wrong scores.
 * The paper has no counterpart: this is a deployment variant of the call above. */
int clusco_crmsd_vs_ref_noalloc(const float *coords, int64_t N, int64_t L, const float *ref, float *out,
                                void *stream);

/* Adjoint of the all-pairs matrix for a loss with dLoss/dcRMSD_ab = grad_out[idx(a,b)]:
 *   grad_coords[a][i] = sum_{b != a} grad_out_ab (a_i - R_ab b_i) / (L max(c_ab, eps))
 * with R_ab the optimal rotation of centred b onto centred a (recomputed, never
 * stored) and c_ab = crmsd[idx] (the forward output, reused). grad_coords is
 * float[N][L][3], overwritten. eps > 0 guards cRMSD -> 0. Pairs with
 * c_ab below the near-duplicate threshold (0.5 A) use a direct FP64 residual path, whose two
 * contributions per pair are added with float atomics: their order, and so the last bits of
 * the gradients of models in such pairs, can differ between runs.
 * On an sm_103 device with L <= 1024 the covariances (three FP16 passes) and the contraction
 * with the rotations (three FP16 passes) run on the tensor cores, in thread-block clusters that
 * compute each rotation once; the form argument is then not used. Otherwise (other devices,
 * larger L) an FP32 CUDA-core path runs. Setting the environment variable
 * CLUSCO_BACKWARD_CLUSTERS=0 makes the tensor-core path run without clusters (each CTA of a
 * row tile recomputes the rotations; same results), for comparison.
 * No counterpart in the paper, which gives no gradient. */
int clusco_crmsd_allpairs_backward(const float *coords, int64_t N, int64_t L, const float *grad_out,
                                   const float *crmsd, float *grad_coords, float eps, int form,
                                   void *workspace, size_t workspace_bytes, void *stream);

/* Kernel timing for benchmarks (no counterpart in the paper). While enabled, every launch
 * of the all-pairs tensor-core kernel (CLUSCO_KERNEL_PAIRS), of the adjoint kernel
 * (CLUSCO_KERNEL_ADJOINT), of the dRMSD tensor-core kernel (CLUSCO_KERNEL_DRMSD) or of the
 * contact-map tensor-core kernel (CLUSCO_KERNEL_CMO) is bracketed by two CUDA events recorded on the launch's own
 * stream. clusco_profile_enable(1) starts a fresh window (unread brackets are dropped),
 * clusco_profile_enable(0) stops recording. clusco_profile_read waits for the kernel's
 * recorded brackets, returns their summed duration (ms) and count, and frees them.
 * Host-side state shared by all threads; EINVAL for an unknown kernel id or null output. */
#define CLUSCO_KERNEL_PAIRS 0
#define CLUSCO_KERNEL_ADJOINT 1
#define CLUSCO_KERNEL_DRMSD 2
#define CLUSCO_KERNEL_CMO 3
int clusco_profile_enable(int on);
int clusco_profile_read(int kernel, double *total_ms, long long *launches);

/* The all-pairs matrix as clusco_crmsd_allpairs, plus each pair's optimal rotation for the
 * adjoint: rot is float[N(N-1)/2][CLUSCO_ROT_STRIDE] (device, caller-owned, 16-byte aligned),
 * in the output's condensed order; rot[idx*CLUSCO_ROT_STRIDE + 3*i + j] = R_ab[i][j], the
 * rotation of centred b onto centred a (natural axis order), which maximises
 * sum_i a_i . R b_i; the record's last three floats are zero (48-byte records). R is dSigma/dM of the eq. 2 sum
 * Sigma (see clusco_crmsd_allpairs_backward_rot), FP32. Tensor-core forms only
 * (CLUSCO_EUNSUPPORTED for CLUSCO_FORM_FP32_SIMT); workspace: CLUSCO_OP_ALLPAIRS_ROT bytes
 * (the all-pairs workspace plus a list of the ~0.5% of pairs whose rotation is solved by
 * Jacobi sweeps after the main kernel).
 * No counterpart in the paper, which needs no rotation. */
#define CLUSCO_ROT_STRIDE 12
int clusco_crmsd_allpairs_rot(const float *coords, int64_t N, int64_t L, float *out, float *rot, int form,
                              void *workspace, size_t workspace_bytes, void *stream);

/* The adjoint of clusco_crmsd_allpairs_backward from the rotations a clusco_crmsd_allpairs_rot
 * call stored (rot, same ensemble and order): no covariance or rotation is recomputed, so the
 * call only gathers R_ab, c_ab and grad_out_ab and contracts on the tensor cores. Same result,
 * tolerance and near-duplicate handling as clusco_crmsd_allpairs_backward. L <= 512 and an
 * sm_103 device (else CLUSCO_EUNSUPPORTED); workspace: CLUSCO_OP_BACKWARD_ROT bytes.
 * No counterpart in the paper, which gives no gradient. */
int clusco_crmsd_allpairs_backward_rot(const float *coords, int64_t N, int64_t L, const float *grad_out,
                                       const float *crmsd, const float *rot, float *grad_coords, float eps,
                                       void *workspace, size_t workspace_bytes, void *stream);

/* One training step of the all-pairs matrix in one call: clusco_crmsd_allpairs_rot (out, rot)
 * followed by clusco_crmsd_allpairs_backward_rot of the weights grad_out (grad_coords), with the
 * same arguments, results and limits as those two calls made in turn. The adjoint's pre-pass
 * reads only coords and grad_out, so the call runs it on a stream of the library's own (one per
 * host thread and device, created on the thread's first fused call and kept until the process
 * exits), forked from and joined back into stream by events, beside the forward. grad_out must therefore be final when the call is
 * made (its values may not depend on this call's out). Every kernel is ordered after the work
 * already enqueued on stream, and every later work on stream after the call's. Calls from
 * several host threads never share a side stream. Workspace: CLUSCO_OP_STEP_ROT bytes (the two calls' workspaces,
 * each 256-byte aligned). No counterpart in the paper, which gives no gradient. */
int clusco_crmsd_allpairs_step_rot(const float *coords, int64_t N, int64_t L, const float *grad_out, float *out,
                                   float *rot, float *grad_coords, int form, float eps, void *workspace,
                                   size_t workspace_bytes, void *stream);

/* One training step in one call, nothing stored between its halves: clusco_crmsd_allpairs (out)
 * followed by clusco_crmsd_allpairs_backward of the weights grad_out (grad_coords), with the same
 * arguments, results and limits as those two calls made in turn; tensor-core forms only,
 * L <= 1024 (else CLUSCO_EUNSUPPORTED). The adjoint's pre-pass reads only coords and grad_out, so
 * the call runs it on a stream of the library's own, one per host thread and device (created on
 * the thread's first fused call, kept until the process exits), forked from and joined back into
 * stream by events, beside the forward. grad_out must therefore be final when the call is made (its
 * values may not depend on this call's out). Every kernel is ordered after the work already
 * enqueued on stream, and every later work on stream after the call's. With a workspace given,
 * the call can be captured into a CUDA graph from stream (the fork and the join become edges of
 * the graph); while that capture is open the thread's side stream belongs to it, so the thread
 * makes no uncaptured fused call until the capture ends. Workspace: CLUSCO_OP_STEP bytes (the
 * two calls' workspaces, each 256-byte aligned). No counterpart in the paper, which gives no
 * gradient. */
int clusco_crmsd_allpairs_step(const float *coords, int64_t N, int64_t L, const float *grad_out, float *out,
                               float *grad_coords, int form, float eps, void *workspace, size_t workspace_bytes,
                               void *stream);

/* Synchronise stream, return the device status word (CLUSCO_OK if clean) and clear it. */
int clusco_sync_status(void *stream);

/* Thread-local message for the last non-OK return of this thread ("" if none). */
const char *clusco_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLUSCO_H */
