/*
 * swmm.h -- C ABI of the GB300 (sm_103a) Strassen / Strassen-Winograd matrix product.
 *
 * Every entry point computes C <- A * B (overwrite; no alpha/beta), the problem of
 * Sec. 2.1 of arXiv 2309.00628 ("Algoritmos para Multiplicacao Matricial"):
 *   c_ij = sum_p a_ip b_pj,  C m x n,  A m x k,  B k x n  (the Sec. 3.4 naming).
 * Matrices are ROW-MAJOR with leading dimensions (elements): A[i*lda + p],
 * B[p*ldb + j], C[i*ldc + j].  A column-major caller gets the same product by
 * passing the transposed problem (C^T = B^T A^T).
 *
 * Pointers:  device pointers unless the name says _host.  The caller owns A, B and C
 * and the stream; the library owns its workspace (taken from the budget given to
 * sw_create) and never frees caller memory.  Calls are asynchronous on `stream`
 * (a cudaStream_t passed as void*, NULL = legacy default stream) unless documented
 * otherwise; device-side failures (a bounded wait that expired) are reported by
 * sw_sync().  No call throws; every call returns an sw_status, and sw_last_error()
 * gives a one-line reason for the last non-OK status on the handle.
 *
 * Variant bitfield (OR one value of each group):
 *   algorithm   SW_ALGO_NAIVE     plain product (Alg. 1) as one tiled tensor-core GEMM
 *               SW_ALGO_STRASSEN  Strassen's 7 products and 18 additions (Sec. 2.2, Alg. 2)
 *               SW_ALGO_WINOGRAD  Strassen-Winograd, the 22-operation BDPZ form (Sec. 2.3, Alg. 3)
 *               SW_ALGO_WINOGRAD_KNUTH  Strassen-Winograd in Knuth's form (Sec. 2.3: u, v, w with
 *                                 aA, bB, (a+b-c-d)D, d(B+C-A-D)), the form the paper implemented;
 *                                 the same seven products, operand sums grouped as Knuth writes
 *                                 them (FUSED schedule only)
 *   schedule    SW_SCHED_FUSED    all levels' operand sums in one pass; the 7^L leaf products in
 *                                 one grouped launch whose epilogue adds +-P into the C blocks
 *                                 (at most 3 levels; FP64 Strassen / BDPZ products go deeper by
 *                                 Alg. 2 / Table 2 steps above a fused 3-level bottom, one per
 *                                 exact halving of m, n, k while the bottom's smallest side stays
 *                                 >= 1024, at most 6 levels)
 *               SW_SCHED_TWO_TEMP Table 2 ("Two Temp Winograd", Sec. 3.3): two temporaries X, Y
 *                                 per level; products written into C quadrants (Winograd only)
 *               SW_SCHED_IN_PLACE Table 3 ("In-Place Winograd", Sec. 3.3): temporaries stored in
 *                                 A, B and C; needs m == n == k; A AND B ARE OVERWRITTEN with
 *                                 unspecified values (Winograd only)
 *               SW_SCHED_ALLOC    Alg. 2 / Alg. 3 as written: fresh temporaries at every level
 *   odd sizes   SW_PAD            zero padding to a multiple of 2^L (Sec. 3.1); virtual (TMA
 *                                 out-of-bounds fill) where the schedule allows, else a copy
 *               SW_PEEL           peel the trailing rows / columns / inner indices that are not a
 *                                 multiple of the split granularity and fix them up with thin
 *                                 products
 *   leaf        SW_LEAF_TF32      FP32 inputs, TF32 tensor-core products (the tensor core reads
 *                                 each FP32 operand as TF32, keeping its 10 leading mantissa
 *                                 bits), FP32 accumulation
 *               SW_LEAF_BF16X3    FP32 inputs split as hi = bf16(x), lo = bf16(x - hi); products
 *                                 hi*hi + hi*lo + lo*hi with FP32 accumulation (FP32-level accuracy)
 *               SW_LEAF_TF32X3    FP32 inputs split as hi = tf32(x) (nearest, ties away), lo = x - hi
 *                                 (FP32, read by the tensor core as TF32); TF32 products
 *                                 lo*hi + hi*lo + hi*hi with FP32 accumulation: a finer operand
 *                                 split than SW_LEAF_BF16X3 at half its tensor rate (on uniform
 *                                 data both reach the FP32-accumulation floor)
 *               SW_LEAF_F64_WTILE FP64 entry points only, with the Winograd algorithms: the FP64
 *                                 leaf GEMM takes one more Winograd step inside each 64 x 64 output
 *                                 tile (its 2 x 2 blocks of 32 x 32; the inner dimension split into
 *                                 the first and last 8 indices of every 16-deep block), with the
 *                                 operand sums formed in shared memory: 7/8 of the leaf's FP64
 *                                 multiply-adds (a register-level base case, like the paper's
 *                                 unrolled small Winograd products, Sec. 3.2).  SW_EINVAL on the
 *                                 FP32 entries, SW_EUNSUPPORTED with SW_ALGO_NAIVE / STRASSEN.
 *   The FP64 entry points ignore the FP32 leaf kinds (TF32, BF16X3, TF32X3): their leaves are FP64.
 *
 * Recursion depth L (Sec. 3.4 cutoff): halve while min(ceil(m/2^l), ceil(n/2^l), ceil(k/2^l))
 * > cutoff.  SW_ALGO_NAIVE ignores the cutoff.  cutoff <= 0 asks the library's autotuner: the
 * first call for a shape (a problem list for sw_mm_batched) and variant times the candidate depths
 * (batched: also the grouped GEMM's tile shape) on the caller's operands, keeps the fastest and
 * runs it once more, so C holds exactly its result; later calls reuse the decision (per handle).
 * That first call therefore runs the product several times and waits for the stream.  Under stream
 * capture, and for SW_SCHED_IN_PLACE (whose runs overwrite A and B), a static default applies
 * instead (FP32: cutoff 8192; FP64: 128), which is also what sw_mm_depth reports for cutoff <= 0.
 */
#ifndef SWMM_H
#define SWMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SW_OK = 0,
    SW_EINVAL = 1,        /* bad argument (negative size, null pointer, ld too small, ...) */
    SW_ENOMEM = 2,        /* device allocation failed */
    SW_EBUDGET = 3,       /* the request needs more workspace than the handle's budget */
    SW_ECUDA = 4,         /* a CUDA runtime / driver call failed */
    SW_ETIMEOUT = 5,      /* a bounded device-side wait expired (see sw_sync) */
    SW_EUNSUPPORTED = 6   /* valid request the library does not implement (e.g. IN_PLACE, m != n) */
} sw_status;

#define SW_ALGO_NAIVE 0x0u
#define SW_ALGO_STRASSEN 0x1u
#define SW_ALGO_WINOGRAD 0x2u
#define SW_ALGO_WINOGRAD_KNUTH 0x3u
#define SW_ALGO_MASK 0xFu
#define SW_SCHED_FUSED 0x00u
#define SW_SCHED_TWO_TEMP 0x10u
#define SW_SCHED_IN_PLACE 0x20u
#define SW_SCHED_ALLOC 0x30u
#define SW_SCHED_MASK 0xF0u
#define SW_PAD 0x000u
#define SW_PEEL 0x100u
#define SW_ODD_MASK 0xF00u
#define SW_LEAF_TF32 0x0000u
#define SW_LEAF_BF16X3 0x1000u
#define SW_LEAF_TF32X3 0x2000u
#define SW_LEAF_F64_WTILE 0x3000u
#define SW_LEAF_MASK 0xF000u

typedef struct sw_handle_s *sw_handle;

/* Create a handle on the current CUDA device.  `workspace_budget_bytes` caps the device
 * memory the library may hold for temporaries (0 = no cap).  Memory is taken lazily.
 * A handle's workspace, cached plans and host-operand buffers serve all its products: issue the
 * products of one handle from one host thread at a time and on one stream (or order the streams
 * yourself); use one handle per stream for independent concurrent work.  The serving calls
 * (sw_server_*) are the exception and may be used from any thread. */
sw_status sw_create(sw_handle *h, size_t workspace_budget_bytes);

/* Release the handle and all memory it holds.  Synchronises the device first. */
sw_status sw_destroy(sw_handle h);

/* One-line reason for the last non-OK status returned on `h` ("" if none). */
const char *sw_last_error(sw_handle h);

/* Workspace bytes the product would take (elem_bytes 4 = FP32 entry, 8 = FP64 entry),
 * without running it.  For SW_SCHED_ALLOC this is the peak of the per-level temporaries
 * (Alg. 3: 4 S + 4 T + 7 P blocks per level, all levels live); for SW_SCHED_TWO_TEMP the
 * X and Y temporaries of every level (Table 2); SW_SCHED_IN_PLACE needs none beyond a
 * padded copy for unaligned sizes; SW_SCHED_FUSED the materialised operand sums (deep FP64
 * products: those of one fused three-level bottom plus the Table 2 X, Y of the levels above). */
sw_status sw_mm_workspace_size(int m, int n, int k, int cutoff, uint32_t variant, int elem_bytes,
                               size_t *bytes);

/* Recursion depth the product will use (see the header comment). */
sw_status sw_mm_depth(int m, int n, int k, int cutoff, uint32_t variant, int elem_bytes, int *depth);

/* FP32 product C <- A B (device pointers, row-major).  Asynchronous on `stream`.
 * Alignment: fastest when A, B, C are 16-byte aligned and lda, ldb, ldc are multiples of 4;
 * otherwise the operands are copied into aligned workspace first. */
sw_status sw_smm(sw_handle h, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                 int m, int n, int k, int cutoff, uint32_t variant, void *stream);

/* FP64 product C <- A B (device pointers, row-major); FP64 leaves and additions. */
sw_status sw_dmm(sw_handle h, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                 int m, int n, int k, int cutoff, uint32_t variant, void *stream);

/* Part of a product for a split of the top recursion level over several GPUs.  The seven products
 * of one Strassen or Strassen-Winograd level (Sec. 2.2 P1..P7; Sec. 2.3 P1..P7, Knuth's form in the
 * same numbering) are independent: a rank computes some of them and the ranks' results are summed.
 * This call overwrites C (device pointer, elem_bytes 4: FP32 as sw_smm, 8: FP64 as sw_dmm) with the
 * contributions to A B of the top-level products whose bit is set in product_mask (bit i = product
 * i + 1), everything below the top level computed as sw_smm / sw_dmm would; C blocks that none of
 * them reaches are zero.  The results of masks that partition 0x7F add up to A B (exactly on
 * small-integer inputs).  Needs SW_SCHED_FUSED, a Strassen or Winograd algorithm and a recursion
 * depth of 1 to 3 (else SW_EUNSUPPORTED); cutoff <= 0 takes the static default (no tuning).
 * Asynchronous on `stream`.  The summation across GPUs is the caller's (a reduction of C). */
sw_status sw_mm_products(sw_handle h, int elem_bytes, const void *A, int lda, const void *B, int ldb, void *C,
                         int ldc, int m, int n, int k, int cutoff, uint32_t variant, uint32_t product_mask,
                         void *stream);

/* FP32 product with HOST operands: copies A and B to the device, runs sw_smm and copies C back;
 * returns after the work has finished (synchronous).  Pinned host memory gives the fastest
 * copies.  Device buffers come from the handle's workspace.  Large products (n, k >= 1024, at
 * least two row panels, 64 MB of operands) of the FUSED schedule or the naive algorithm with
 * cutoff > 0 move A and C in row panels on two library streams ordered after `stream`: B goes
 * first, then panel i of A; C's panel i = A_i B runs on `stream` at the whole product's depth and
 * comes back while later panels still arrive (the panels' Winograd block partitions differ from
 * one whole-matrix call, so the rounding can differ from sw_smm's within the same bound). */
sw_status sw_smm_host(sw_handle h, const float *A_host, int lda, const float *B_host, int ldb,
                      float *C_host, int ldc, int m, int n, int k, int cutoff, uint32_t variant,
                      void *stream);

/* Self-test of the bounded device waits (failure detection without a GPU fault): launches one
 * small leaf-GEMM whose only contribution is a reduce-add ordered after a first write that no leaf
 * makes, so its epilogue's wait on the ordering counter expires after the bound (about 2 s); the
 * kernel records the expiry, finishes and releases its resources.  Returns what sw_sync reports,
 * SW_ETIMEOUT when the bound works.  The handle and the CUDA context stay usable.  Synchronous. */
sw_status sw_selftest_expired_wait(sw_handle h, void *stream);

/* Wait for `stream` and report device-side failures of this handle's kernels: SW_ETIMEOUT if a
 * bounded wait inside a kernel expired, SW_ECUDA if the stream reported a CUDA error.
 * Clears the device error word. */
sw_status sw_sync(sw_handle h, void *stream);

/* One product of a batch: C <- A B, FP32, row-major, device pointers. */
typedef struct {
    const float *A;
    int lda;
    const float *B;
    int ldb;
    float *C;
    int ldc;
    int m, n, k;
} sw_problem;

/* `count` independent FP32 products (different shapes allowed, any alignment), asynchronous on
 * `stream`.  The tensor-core work of all products runs as ONE persistent grouped launch; the
 * per-product staging (packing operands whose rows are not 16-byte aligned) runs as one batched
 * launch, and depth >= 1 products add their operand-sum passes.  The whole batch is captured once into a CUDA
 * graph and replayed on later calls with the same problem list (same pointers and shapes).
 * Variant: SW_SCHED_FUSED with SW_LEAF_TF32 (other schedules / leaves: SW_EUNSUPPORTED); each
 * product's depth follows `cutoff` as for sw_smm (<= 0: the autotuner picks one cutoff and the tile
 * shape for the whole list).  Odd sizes are padded virtually (TMA out-of-bounds fill). */
sw_status sw_mm_batched(sw_handle h, int count, const sw_problem *probs, int cutoff, uint32_t variant,
                        void *stream);

/* The autotuner's last decision on this handle (a call with cutoff <= 0 that had to tune): the
 * chosen cutoff (1 << 30: no recursion), the grouped GEMM's tile width and CTA-pair flag (batched
 * calls; 0 for single products: 0 one CTA per tile, 1 CTA pairs, 2 CTA pairs whose GEMM launch
 * also runs the copies that pack operands with rows not 16-byte aligned), the winner's device time
 * in ms and the number of candidates timed.
 * Any pointer may be NULL.  SW_EINVAL if nothing has been tuned on the handle. */
sw_status sw_last_tuning(sw_handle h, int *cutoff, int *tile_n, int *cta_pair, double *ms, int *candidates);

/* ---------------------------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Requests (FP32 or FP64 products of any
 * shape) are admitted in arrival order as soon as a completion slot and enough of the serving
 * arena are free -- also while earlier requests are still running -- and their work overlaps on
 * the device.  An FP32 request with TF32 leaves whose plan ends in a grouped leaf GEMM (NAIVE and
 * FUSED schedules on 16-byte aligned operands; the last product of the step-by-step schedules)
 * runs that GEMM inside one device-resident loop: a persistent kernel on `sm_share` SMs that picks
 * up newly published tiles while it runs and exits after `idle_us` without work.  Its staging passes
 * (B^T, operand sums), FP64 requests, split-BF16 leaves and padded or peeled shapes run on side
 * streams with the SMs the loop leaves free.  A request's result is the same alone and in a mix
 * (within the tolerance of its leaf precision; bit-identical for the resident TF32 form, whose
 * tile sums do not depend on the schedule).  The paper has no serving loop: this is the deployment
 * form of the same products.
 *
 * Threading: submit and wait may be called from any thread.  The loop runs on a thread of its own
 * and uses its own streams, so inputs must be complete on the device when submit is called (the
 * caller synchronises the stream that wrote them) and C may be read once wait returned SW_OK.
 * Requests in flight together must not write memory another one reads or writes.  The arena is
 * allocated at start and is separate from the handle's workspace budget.  When a bounded device
 * wait expires every request in flight fails with SW_ETIMEOUT and the loop carries on; a CUDA error
 * fails all current and later requests with SW_ECUDA.
 */
typedef struct {
    int sm_share;        /* SMs (persistent CTAs) of the resident loop; 0: all but 16 */
    int max_inflight;    /* requests admitted at once; 0: 64 */
    size_t budget_bytes; /* workspace the admitted requests may hold together; 0: 60 GB or 3/4 of
                            the free device memory, whichever is less */
    int idle_us;         /* the resident loop exits after this long without new work; 0: 20000 */
} sw_server_cfg;

typedef struct {
    int elem_bytes;      /* 4: FP32 product as sw_smm; 8: FP64 product as sw_dmm */
    const void *A;
    int lda;
    const void *B;
    int ldb;
    void *C;
    int ldc;
    int m, n, k;
    int cutoff;
    uint32_t variant;
} sw_request;

/* Start the serving loop on the handle (one per handle).  NULL cfg: defaults. */
sw_status sw_server_start(sw_handle h, const sw_server_cfg *cfg);
/* Queue a request; the caller keeps A, B and C alive and untouched until sw_server_wait returns
 * for its ticket.  The workspace is sized here, on the caller's thread: SW_EBUDGET if the request
 * alone needs more than the arena; SW_EINVAL / SW_EUNSUPPORTED for arguments sw_smm would refuse. */
sw_status sw_server_submit(sw_handle h, const sw_request *req, uint64_t *ticket);
/* Wait up to timeout_ns (< 0: no limit) for a ticket: SW_OK once C holds the result, SW_ETIMEOUT if
 * it is not done yet (the ticket stays valid), or the request's own failure status. */
sw_status sw_server_wait(sw_handle h, uint64_t ticket, int64_t timeout_ns);
/* Finish every queued request, stop the loop and release its resources (tickets not yet collected
 * become invalid).  sw_destroy stops a running loop the same way. */
sw_status sw_server_stop(sw_handle h);

/* Reductions used by the error checks, FP64 on the device (Sec. 2.1 problem's error metric):
 *   out[0] = max_ij |C_ij - R_ij|,  out[1] = max |A|,  out[2] = max |B|
 * C is FP32 (elem_bytes 4) or FP64 (8); A and B have the same type as C; R is FP64.
 * Any pointer may be NULL (its entry is then 0).  Synchronous: `out` is a host array. */
sw_status sw_error_norms(sw_handle h, int elem_bytes, int m, int n, int k, const void *A, int lda,
                         const void *B, int ldb, const void *C, int ldc, const double *R, int ldr,
                         double *out, void *stream);

/* Measurement support.  While profiling is on, every kernel the library launches is bracketed by
 * a pair of CUDA events on its launch stream.  sw_profile_read() waits for them and returns, per
 * kernel kind, the number of launches and the summed device time in milliseconds since the last
 * read (then resets).  Kinds: 0 tensor-core leaf GEMM (TF32), 1 SIMT leaf GEMM, 2 block addition,
 * 3 padded copy, 4 operand-sum pass, 5 memset, 6 transpose, 7 in-place transpose, 8 bf16 split,
 * 9 tensor-core leaf GEMM (split BF16), 10 batched copy / transpose (sw_mm_batched staging),
 * 11 tf32 split, 12 tensor-core leaf GEMM (compensated TF32), 13 operand sums with split-BF16 output.
 * `nkinds` is the length of both output arrays (entries beyond 14 are set to 0). */
#define SW_PROFILE_KINDS 14
sw_status sw_profile(sw_handle h, int enable);
sw_status sw_profile_read(sw_handle h, int nkinds, int *launches, double *ms);

/* No-allocation product.  The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory: runtimes that reserve nearly all HBM for their
 * own pool at start-up (a library cudaMalloc would fail or fragment it), deployments that forbid
 * device allocation after initialisation, and streams that must not see the implicit
 * synchronisation of cudaMalloc / cudaFree.  It needs no handle and calls no allocating routine.
 *
 * Computes C <- A B (FP32, row-major) with one Strassen-Winograd level in the FUSED schedule and
 * TF32 leaves -- the same operand sums and leaf products as sw_smm with SW_ALGO_WINOGRAD |
 * SW_SCHED_FUSED at depth 1; the seven products are added into a zeroed C with atomic adds in the
 * order they finish, so float results can differ in their last bits from call to call.
 * The caller provides A, B and C; every temporary (B^T, the S and T sums, descriptors, the error
 * word) lives in one static device array of SW_NOALLOC_SCRATCH_BYTES, which every GPU that loads
 * this code holds until the process exits.  A problem fits when
 *   4 * (n * ceil4(k) + 4 * ceil(m/2) * kb + 4 * ceil4(ceil(n/2)) * kb) + ~2 KiB <= 32 MiB,
 *   kb = ceil32(ceil(k/2))   (square problems up to n of about 1670);
 * larger problems return SW_EBUDGET without touching memory.
 * Requirements: m, n, k >= 2; A and C 16-byte aligned; lda and ldc multiples of 4 (else SW_EINVAL).
 * The call is synchronous: it waits for `stream` and returns SW_ETIMEOUT if a bounded device wait
 * expired, SW_ECUDA on a CUDA error.  The first call on a device does a one-time set-up with that
 * device current: it looks up the array's device address and loads the kernels the call uses.
 * With CUDA's default lazy module loading that set-up is when the array (and the kernels' code)
 * take their device memory; later calls take none.  A caller that reserves the GPU's memory for
 * itself should therefore make its first call before reserving (or run with
 * CUDA_MODULE_LOADING=EAGER, which places them when the context is created), and before any stream
 * capture.  All calls share the one array and overwrite it: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
#define SW_NOALLOC_SCRATCH_BYTES (32u << 20)
sw_status sw_smm_noalloc(const float *A, int lda, const float *B, int ldb, float *C, int ldc, int m, int n,
                         int k, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SWMM_H */
