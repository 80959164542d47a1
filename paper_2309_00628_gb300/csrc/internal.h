// internal.h -- launchers shared between the kernels and the host planner (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "plan.h"

namespace swk {

// Tensor maps passed by value (__grid_constant__): A, B and the two operand-sum scratch
// matrices of one product -- one map each for TF32, a (hi, lo) pair each for BF16X3.
struct MapSet {
    CUtensorMap m[8];
};

// A strided matrix view with its valid extent (reads beyond it return 0).
struct MatRef {
    const void* p;
    long long ld;
    int rows, cols;
};

// Leaf for the pointer-based (FP64) kernels: operands are MatRef indices.
// tmaps: tensor maps of the target blocks (Target::map indexes it), or nullptr for the
// per-thread epilogue only.  flags / epoch: the ordering counters of the targets (Target::flag_base)
// and this launch's epoch (1, 2, ... per counter array), or nullptr.
// pair: the CTA-pair form (cta_group::2, 256 x 256 tiles, bn must be 256): work items count
// 256-row tiles (Leaf::tile_begin in those units), B maps have 128-row boxes, `grid` is the number
// of SMs to use (rounded down to whole pairs).  item_leaf: optional device table of the leaf of
// every work item (saves the per-tile binary search over the leaves; nullptr: search).
cudaError_t launch_gemm_tf32(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                             const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                             int total_items, int* err, int grid, cudaStream_t stream, bool pair = false,
                             const int* item_leaf = nullptr);
// The batched TF32N CTA-pair launch that also packs operands: jobs[0..njobs) (CopyJob::pad_ = its
// tile count of BCOPY_TILE x BCOPY_TILE, tile_begin its first tile of pack_tiles) write the packed
// copies its leaves' maps read; flags holds the launch epoch and one counter per job.
cudaError_t launch_gemm_tf32n_pack(const CUtensorMap* gmaps, const Leaf* leaves, int nleaves, const Target* targets,
                                   const CUtensorMap* tmaps, unsigned* flags, int total_items, int* err, int grid,
                                   cudaStream_t stream, const int* item_leaf, const CopyJob* jobs, int njobs,
                                   int pack_tiles);
// TF32 leaves with B N-major (k x n as stored; maps from make_map_f32_n, Leaf::b_row = K,
// Leaf::b_col = N); otherwise as launch_gemm_tf32.  bn = 512 (CTA pairs only): 256 x 512 tiles with
// one TMEM accumulator.
// item_tile / units: an explicit work layout (tile row << 16 | column per item, with item_leaf its
// leaf) planned for exactly `units` persistent units; the launch uses that many (accumulation
// chains rely on unit u taking items u, u + units, ...).
cudaError_t launch_gemm_tf32n(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                              const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                              int total_items, int* err, int grid, cudaStream_t stream, bool pair = false,
                              const int* item_leaf = nullptr, const int* item_tile = nullptr, int units = 0);
// Persistent units (CTA pairs) of a pair-form N-major TF32 launch with tile width bn (256 or
// 512) on `sms` SMs (0: unavailable).
int gemm_tf32n_pair_units(int sms, int bn = 256);
// Resident (serving) form of the TF32 grouped GEMM, BN = 256: runs until ctl.stop, an error, or
// ctl.idle_ns without newly published items.  nmajor: B maps N-major (as launch_gemm_tf32n), else B^T.
cudaError_t launch_gemm_tf32_resident(const CUtensorMap* gmaps, const Leaf* leaves, const Target* targets,
                                      const CUtensorMap* tmaps, const ResidentCtl& ctl, int* err, int grid,
                                      cudaStream_t stream, bool nmajor);
// Load the one-CTA, non-resident B^T-form TF32 kernels (tile widths 128 and 256) into device memory
// now and set their shared-memory attribute; with lazy module loading they would be loaded at
// their first launch.
cudaError_t preload_gemm_tf32();
int tf32_tile_m();
int tf32_tile_k();
int bf16x3_tile_k();

// Split-BF16 leaves: operand map index i refers to maps 2i (hi) and 2i+1 (lo); B is N-major
// (k x n as stored); Leaf::kblocks counts 64-deep k blocks.
cudaError_t launch_gemm_bf16x3(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                               const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                               int total_items, int* err, int grid, cudaStream_t stream,
                               const int* item_leaf = nullptr, const int* item_tile = nullptr, int units = 0,
                               bool pair = false);
// Persistent units (CTA pairs) of a pair-form split-BF16 launch on `sms` SMs (0: unavailable).
int gemm_bf16x3_pair_units(int sms);

// Compensated-TF32 leaves: operand map index i refers to maps 2i (hi) and 2i+1 (lo), FP32 halves
// with hi = tf32(x), lo = x - hi; A K-major (make_map_f32, 128-row boxes), B N-major
// (make_map_f32_n); Leaf::kblocks counts 32-deep k blocks.
cudaError_t launch_gemm_tf32x3(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                               const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                               int total_items, int* err, int grid, cudaStream_t stream,
                               const int* item_leaf = nullptr);
// hi = tf32(x) (round to nearest, ties away), lo = x - hi (exact), elementwise on a rows x cols
// FP32 view; both outputs FP32 with leading dimension ldo.
cudaError_t launch_split_tf32(int rows, int cols, const float* x, long long ldx, float* hi, float* lo, long long ldo,
                              cudaStream_t stream);

// hi = bf16(x), lo = bf16(x - hi), elementwise on a rows x cols FP32 view; outputs share ldo.
cudaError_t launch_split_bf16(int rows, int cols, const float* x, long long ldx, void* hi, void* lo, long long ldo,
                              cudaStream_t stream);

// SIMT leaf GEMM (FP64, or FP32 when elem_bytes == 4): same leaf / target descriptors,
// a_map / b_map index `refs`, B stored as is (k x n); Leaf::kblocks is the inner dimension.
// wtile (FP64): every 64 x 64 tile takes one Winograd step over its 2 x 2 blocks.
cudaError_t launch_gemm_simt(int elem_bytes, const MatRef* refs, const Leaf* leaves, int nleaves,
                             const Target* targets, int total_items, int grid, bool wtile, cudaStream_t stream);
constexpr int F64_BM = 64, F64_BN = 64;

// out (out_rows x out_cols) <- x^T, zero outside the source extent (src_rows x src_cols).
cudaError_t launch_transpose_pad(int out_rows, int out_cols, float* out, long long ldo, const float* x,
                                 long long ldx, int src_rows, int src_cols, cudaStream_t s);
// Load the kernels launch_transpose_pad may launch and the FP32 depth-1 BDPZ operand-sum kernels
// of launch_preadd (A side, and B side held as B^T; vector and scalar forms) into device memory now.
cudaError_t preload_transpose_preadd_f32_l1();
// x (n x n view) <- x^T in place.
cudaError_t launch_transpose_inplace(int n, float* x, long long ld, cudaStream_t s);

// Z = X + sy * Y elementwise on strided views (FP32 or FP64 per elem_bytes).
cudaError_t launch_addsub(int elem_bytes, int rows, int cols, void* z, long long ldz, const void* x, long long ldx,
                          const void* y, long long ldy, float sy, cudaStream_t stream);

// Two independent elementwise jobs z = x + sy * y (FP32 or FP64 per elem_bytes) in one launch.
struct AddJob {
    int rows, cols;
    void* z;
    long long ldz;
    const void* x;
    long long ldx;
    const void* y;
    long long ldy;
    float sy;
    // FP32 only, optional: z's bf16 halves hi = bf16(z), lo = bf16(z - hi) (leading dimension ldh),
    // written in the same pass for split-BF16 leaves that read z next
    void* zh = nullptr;
    void* zl = nullptr;
    long long ldh = 0;
};
cudaError_t launch_addsub2(int elem_bytes, const AddJob& a, const AddJob& b, cudaStream_t stream);

// Z = X (strided 2-D copy with zero fill outside the source extent).
cudaError_t launch_copy_pad(int elem_bytes, int rows, int cols, void* z, long long ldz, const void* x,
                            long long ldx, int src_rows, int src_cols, cudaStream_t stream);

// One pass over a 2^L x 2^L grid of blocks of X that writes every non-pure leaf operand sum
// (all recursion levels at once) into `out` (slot s occupies rows [s*brows, (s+1)*brows),
// leading dimension bcols).  bside: B-side coefficients.
struct PreaddArgs {
    const void* x;
    long long ldx;
    int rows, cols;      // real extent of X
    int brows, bcols;    // leaf block extent
    void* out;
    int L, alg, bside;   // alg: 1 Strassen, 2 Winograd (BDPZ), 3 Winograd (Knuth form)
    int bt;              // B side stored as B^T (quadrants 12 and 21 swap roles)
    short slot_of[343];  // leaf word -> output slot, -1 = pure (not written)
};
cudaError_t launch_preadd(int elem_bytes, const PreaddArgs& a, cudaStream_t stream);
// Operand sums with split-BF16 output (depth 1 or 2, FP32 vector path, X as stored), both sides
// in one launch: writes the bf16 halves of X (xh / xl, leading dimension ldx_out, a multiple of 8)
// and of every sum slot (sh / sl, slot s at element s * brows * bcols, row stride bcols, a
// multiple of 8); 16-byte aligned buffers.
struct PreaddSplitOut {
    __nv_bfloat16* xh;
    __nv_bfloat16* xl;
    long long ldx_out;
    __nv_bfloat16* sh;
    __nv_bfloat16* sl;
};
cudaError_t launch_preadd_split(const PreaddArgs& a, const PreaddSplitOut& oa, const PreaddArgs& b,
                                const PreaddSplitOut& ob, cudaStream_t stream);

// The A-side (a) and B-side (b) passes of one FP32 product in a single launch (falls back to two
// launches where the vector path or the shapes do not allow it).
cudaError_t launch_preadd2(const PreaddArgs& a, const PreaddArgs& b, cudaStream_t stream);

// One FP32 copy (or transpose) job of a batched launch: out (out_rows x out_cols) <- x or x^T,
// zero outside the source extent; tile_begin is the job's first BCOPY_TILE x BCOPY_TILE output
// tile (prefix sum).
constexpr int BCOPY_TILE = 64;
struct CopyJob {
    const void* x;
    long long ldx;
    void* out;
    long long ldo;
    int src_rows, src_cols, out_rows, out_cols;
    int tile_begin, pad_;  // pad_: the job's tile count where a GEMM launch packs (else unused)
};
cudaError_t launch_batched_copy(const CopyJob* jobs, int njobs, int total_tiles, int transpose, cudaStream_t s);

// Device reductions for the error metric (results are written to d_out[0..2] as doubles).
cudaError_t launch_norms(int elem_bytes, int m, int n, int k, const void* A, long long lda, const void* B,
                         long long ldb, const void* C, long long ldc, const double* R, long long ldr,
                         unsigned long long* d_out, cudaStream_t stream);

}  // namespace swk
