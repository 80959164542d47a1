// api.cu -- C ABI (include/swmm.h), workspace pool and the planner that lowers a product
// C <- A B into kernel launches:
//
//   NAIVE            one grouped-GEMM launch, one leaf, one STORE target (Alg. 1 on tensor cores)
//   FUSED            one operand-sum pass per operand (all L levels at once) + one grouped-GEMM
//                    launch over the 7^L leaves; the leaf epilogues add +-P into the C blocks
//   TWO_TEMP         Table 2 of Sec. 3.3, step by step, X / Y temporaries per level
//   IN_PLACE         Table 3 of Sec. 3.3, step by step, temporaries in A, B and C
//   ALLOC            Alg. 2 / Alg. 3 as written: fresh temporaries at every level
//
// The recursion depth follows the Sec. 3.4 cutoff; odd sizes are padded (Sec. 3.1) or peeled.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <functional>
#include <unordered_map>
#include <vector>

#include "../../include/swmm.h"
#include "internal.h"
#include "plan.h"
#include "arena.h"

using namespace swk;

namespace {

// ------------------------------------------------------------------ tensor-map encoding
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// FP32 row-major view rows x cols (ld elements) -> 2-D tensor map with a box of
// box_cols (innermost, 128 bytes) x box_rows, 128-byte swizzle, zero fill out of bounds.
bool make_map_f32(CUtensorMap* m, const void* base, int rows, int cols, long long ld, int box_cols, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)std::max(cols, 1), (cuuint64_t)std::max(rows, 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// FP32 row-major k x n view of an N-major B operand (ld elements) -> 2-D tensor map with a box of
// 32 columns (128 bytes) x 32 rows, 128-byte swizzle with 32-byte atoms (the layout the tensor core
// reads an MN-major TF32 operand from), zero fill out of bounds.
bool make_map_f32_n(CUtensorMap* m, const void* base, int rows, int cols, long long ld) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)std::max(cols, 1), (cuuint64_t)std::max(rows, 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// BF16 row-major view rows x cols (ld elements, a multiple of 8) -> 2-D tensor map with a box of
// 64 columns (128 bytes) x box_rows, 128-byte swizzle, zero fill out of bounds.
bool make_map_bf16(CUtensorMap* m, const void* base, int rows, int cols, long long ld, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)std::max(cols, 1), (cuuint64_t)std::max(rows, 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// SWMM_TF32_BT=1: the TF32 leaves read B as B^T (staged by a transpose) instead of N-major as
// stored -- a diagnostics switch; the default is N-major everywhere.
bool tf32_bt_form() {
    static const bool bt = getenv("SWMM_TF32_BT") != nullptr;
    return bt;
}

// Tile-width override for tuning sweeps (SWMM_TF32_BN = 128, 256 or 512); 0 = the planner's choice.
int bn_override() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SWMM_TF32_BN");
        v = e ? atoi(e) : 0;
        if (v != 128 && v != 256 && v != 512) v = 0;
    }
    return v;
}
inline long long ceil_div(long long x, long long a) { return (x + a - 1) / a; }

// ------------------------------------------------------------------ plan
enum OpKind {
    OP_GEMM_TF32, OP_GEMM_SIMT, OP_ADDSUB, OP_COPY_PAD, OP_PREADD, OP_MEMSET, OP_TRANSPOSE, OP_TRANSPOSE_SQ,
    OP_SPLIT, OP_GEMM_BF16X3, OP_BATCH_COPY, OP_SPLIT_TF32, OP_GEMM_TF32X3, OP_PREADD_SPLIT
};

struct Op {
    OpKind kind;
    // grouped GEMM
    MapSet maps;
    int bn = 256, nleaves = 0, items = 0, ntmaps = 0, nflags = 0;
    bool pair = false;   // TF32: the CTA-pair form (256 x 256 tiles; items count 256-row tiles)
    bool has_item_leaf = false;  // tensor-core GEMM: item -> leaf table at item_leaf_off
    bool has_layout = false;     // explicit work layout: item_leaf_off (leaf) and item_tile_off (tile)
    size_t item_tile_off = 0;
    int units = 0;               // the layout's persistent units
    bool nmaj = false;           // TF32 GEMM reading B N-major (launch_gemm_tf32n)
    size_t item_leaf_off = 0;
    size_t leaves_off = 0, targets_off = 0, refs_off = 0, tmaps_off = 0, flags_off = 0;
    int ngmaps = 0, njobs = 0, tiles = 0, transpose = 0;
    size_t gmaps_off = 0, jobs_off = 0;  // operand maps in global memory; batched copy jobs
    // elementwise
    int eb = 4, rows = 0, cols = 0, src_rows = 0, src_cols = 0;
    void* z = nullptr;
    long long ldz = 0, ldx = 0, ldy = 0;
    const void* x = nullptr;
    const void* y = nullptr;
    float sy = 1.f;
    PreaddArgs pre;
    PreaddArgs pre_b;       // FP32: the B side of the same pass (pre_two: one launch for both)
    bool pre_two = false;
    bool wtile = false;     // OP_GEMM_SIMT (FP64): one Winograd step inside every 64 x 64 tile
    PreaddSplitOut sout;    // OP_PREADD_SPLIT: bf16 halves of A and of its sums (sout_b: of B)
    PreaddSplitOut sout_b;
};

struct Plan {
    std::vector<Op> ops;
    std::vector<uint8_t> blob;  // leaves / targets / refs, uploaded once
    void* d_blob = nullptr;
    size_t ws_need = 0;
    int depth = 0;
    bool use_graph = false;               // replay through a captured CUDA graph
    bool owns_blob = true;                // false: d_blob lives in memory the server owns
    cudaGraphExec_t gexec = nullptr;
    ~Plan() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (d_blob && owns_blob) cudaFree(d_blob);
    }
};

// A row-major view (byte pointer, ld in elements).
struct View {
    char* p;
    long long ld;
    int rows, cols;
};

// Lowers one product to ops.  The TF32 leaves read B N-major, as stored (nmaj).  In the B^T
// form (serving plans, SWMM_TF32_BT=1) the tensor cores take B as B^T (K-major), so every
// B-side value -- B itself, its quadrants, the T sums and the B-side temporaries -- is held
// transposed ("bt" storage): a logical B quadrant Bij lives at position ji of the stored
// matrix, and a k x n block is stored n x k.  Elementwise steps are orientation-free as long
// as all their operands share it, which the schedules below guarantee.
struct Planner {
    int eb;                 // 4 = FP32 (TF32 or split-BF16 leaves), 8 = FP64
    bool bf;                // FP32 with split-BF16 leaves
    bool x3 = false;        // FP32 with compensated-TF32 leaves (FP32 hi / lo halves)
    bool wtile = false;     // FP64 leaves: one Winograd step inside every 64 x 64 tile
    int fused_below = 0;    // deep FUSED (FP64): sub-products at this depth or less are fused
    bool bt;                // B side stored transposed (TF32 leaves read through B^T)
    bool nmaj = false;      // TF32 leaves read B N-major, as stored (bt is then false)
    uint32_t variant;
    bool dry;               // size only: no pointers, no maps
    char* ws_base;
    size_t ws_top = 0, ws_peak = 0;
    Plan* plan;
    std::string err;
    int sched, algo;

    // Batch mode: products append their leaves, targets and operand maps to one grouped launch
    // instead of emitting their own (operand maps then live in global memory).
    bool batch = false;
    bool server = false;  // plan for the serving loop (no ordering counters)
    int force_bn = 0;
    int sms = 0;              // SMs of the device (explicit work layouts are planned for its units)
    int batch_bn = 256;       // batched launch: tile width of the grouped GEMM (128 or 256)
    bool batch_pair = false;  // batched launch: CTA-pair form (256 x 256 tiles; N-major B only)
    // The CTA-pair GEMM (cta_group::2; TF32 and split-BF16 leaves) serves single products with
    // 256-wide tiles; batched and serving launches keep the one-CTA form unless told otherwise.
    // SWMM_NO_PAIR=1 disables it (diagnostics).
    bool pair_ok(int bn) const {
        static const bool off = getenv("SWMM_NO_PAIR") != nullptr;
        return !off && (bn == 256 || (bn == 512 && nmaj && !bf)) && !batch && !server && !x3 && eb == 4;
    }
    // Tile width of a TF32 launch over C blocks `cols` wide: 512 (CTA pairs, one accumulator, a
    // quarter fewer operand bytes per MMA) where the blocks are at least 512 wide and 512-wide tiles
    // pad no more than 256-wide ones; else 256, or 128 for narrow blocks.
    int tf32_bn(int cols) const {
        if (bn_override()) return bn_override() == 512 && !pair_ok(512) ? 256 : bn_override();
        if (cols <= 128) return 128;
        if (pair_ok(512) && cols >= 512 && round_up(cols, 512) == round_up(cols, 256)) return 512;
        return 256;
    }
    // rows of one B-side TMA box: half the tile width for a CTA pair
    int b_box(int bn) const { return pair_ok(bn) ? bn / 2 : bn; }
    // Renumber a TF32 op's work items in 256-row tiles for the pair kernel.
    void to_pair(Op& o, std::vector<Leaf>& leaves) const {
        int items = 0;
        for (Leaf& lf : leaves) {
            lf.tile_begin = items;
            items += (int)(ceil_div(lf.m, 2 * tf32_tile_m()) * lf.tiles_n);
        }
        o.items = items;
        o.pair = true;
    }
    std::vector<CUtensorMap> bmaps;
    std::vector<Leaf> bleaves;
    std::vector<Target> btargets;
    int bitems = 0;

    View quad(View v, int q) const {
        const int h = v.rows / 2, w = v.cols / 2;
        View r;
        r.p = v.p + ((long long)(q >> 1) * h * v.ld + (long long)(q & 1) * w) * eb;
        r.ld = v.ld;
        r.rows = h;
        r.cols = w;
        return r;
    }
    // logical quadrant q of a B-side block held in bt storage
    View quadB(View v, int q) const { return quad(v, bt ? (q == 1 ? 2 : q == 2 ? 1 : q) : q); }

    static View sub(View v, long long r0, long long c0, long long rows, long long cols, int eb) {
        View s = v;
        s.p = v.p + (r0 * v.ld + c0) * eb;
        s.rows = (int)rows;
        s.cols = (int)cols;
        return s;
    }

    View talloc(int rows, int cols) {
        const long long ld = round_up(std::max(cols, 1), 4);
        const size_t bytes = (size_t)round_up((long long)std::max(rows, 1) * ld * eb, 256);
        View v;
        v.p = dry ? nullptr : ws_base + ws_top;
        v.ld = ld;
        v.rows = rows;
        v.cols = cols;
        ws_top += bytes;
        ws_peak = std::max(ws_peak, ws_top);
        return v;
    }
    // a logical k x n B-side temporary
    View tallocB(int k, int n) { return bt ? talloc(n, k) : talloc(k, n); }

    // a bf16 rows x cols buffer, leading dimension a multiple of 8 (16-byte TMA rows)
    View talloc_bf16(int rows, int cols) {
        const long long ld = round_up(std::max(cols, 1), 8);
        const size_t bytes = (size_t)round_up((long long)std::max(rows, 1) * ld * 2, 256);
        View v;
        v.p = dry ? nullptr : ws_base + ws_top;
        v.ld = ld;
        v.rows = rows;
        v.cols = cols;
        ws_top += bytes;
        ws_peak = std::max(ws_peak, ws_top);
        return v;
    }

    // one half of a split operand: bf16 (split-BF16 leaves) or FP32 (compensated TF32)
    View talloc_half(int rows, int cols) { return x3 ? talloc(rows, cols) : talloc_bf16(rows, cols); }

    // FP32 view -> (hi, lo) halves in workspace
    void split(View x, View& hi, View& lo) {
        hi = talloc_half(x.rows, x.cols);
        lo = talloc_half(x.rows, x.cols);
        split_into(x, hi, lo);
    }
    void split_into(View x, const View& hi, const View& lo) {
        Op o;
        o.kind = x3 ? OP_SPLIT_TF32 : OP_SPLIT;
        o.rows = x.rows;
        o.cols = x.cols;
        o.x = x.p;
        o.ldx = x.ld;
        o.z = hi.p;
        o.y = lo.p;
        o.ldz = hi.ld;
        push(o);
    }

    size_t put_blob(const void* src, size_t bytes) {
        size_t off = round_up(plan->blob.size(), 64);
        plan->blob.resize(off + bytes);
        if (bytes) memcpy(plan->blob.data() + off, src, bytes);
        return off;
    }

    void push(const Op& o) {
        if (!dry) plan->ops.push_back(o);
    }

    void add(View z, View x, View y, float sy) {
        Op o;
        o.kind = OP_ADDSUB;
        o.eb = eb;
        o.rows = z.rows;
        o.cols = z.cols;
        o.z = z.p;
        o.ldz = z.ld;
        o.x = x.p;
        o.ldx = x.ld;
        o.y = y.p;
        o.ldy = y.ld;
        o.sy = sy;
        push(o);
    }

    void copy_pad(View z, View x) {  // z (its full extent) <- x, zero outside x's extent
        Op o;
        o.kind = OP_COPY_PAD;
        o.eb = eb;
        o.rows = z.rows;
        o.cols = z.cols;
        o.z = z.p;
        o.ldz = z.ld;
        o.x = x.p;
        o.ldx = x.ld;
        o.src_rows = x.rows;
        o.src_cols = x.cols;
        push(o);
    }

    void transpose_into(View z, View x) {  // z (its full extent) <- x^T, zero outside
        Op o;
        o.kind = OP_TRANSPOSE;
        o.eb = 4;
        o.rows = z.rows;
        o.cols = z.cols;
        o.z = z.p;
        o.ldz = z.ld;
        o.x = x.p;
        o.ldx = x.ld;
        o.src_rows = x.rows;
        o.src_cols = x.cols;
        push(o);
    }

    void transpose_square(View z) {
        Op o;
        o.kind = OP_TRANSPOSE_SQ;
        o.eb = 4;
        o.rows = z.rows;
        o.z = z.p;
        o.ldz = z.ld;
        push(o);
    }

    void memset0(View z) {
        Op o;
        o.kind = OP_MEMSET;
        o.eb = eb;
        o.rows = z.rows;
        o.cols = z.cols;
        o.z = z.p;
        o.ldz = z.ld;
        push(o);
    }

    static bool vec_ok(const View& v) {
        return ((reinterpret_cast<uintptr_t>(v.p) & 15) == 0) && (v.ld % 4) == 0;
    }

    static Target make_target(View c, float sign, int mode, int map = -1) {
        Target t;
        t.c = c.p;
        t.ldc = c.ld;
        t.rows = c.rows;
        t.cols = c.cols;
        t.sign = sign;
        t.mode = mode;
        t.vec_ok = vec_ok(c) ? 1 : 0;
        t.map = map;
        t.flag_base = -1;
        t.flag_cols = 0;
        return t;
    }

    // Tensor maps of the target blocks of one GEMM launch (TMA store / reduce-add epilogue),
    // one per distinct block.
    std::vector<CUtensorMap> tmaps;
    std::vector<View> tmap_views;
    // A TMA store / reduce writes whole 16-byte pieces at a block's right edge, so a block whose
    // width is not a multiple of 4 FP32 elements would spill into its right-hand neighbour (or a
    // caller's padding): such blocks keep the per-thread epilogue.
    int target_map(View c) {
        static const bool no_tma_epilogue = getenv("SWMM_NO_TMA_EPILOGUE") != nullptr;  // diagnostics
        if (eb != 4 || no_tma_epilogue || !vec_ok(c) || c.rows <= 0 || c.cols <= 0 || (c.cols % 4) != 0)
            return -1;
        for (size_t i = 0; i < tmap_views.size(); ++i) {
            const View& v = tmap_views[i];
            if (v.p == c.p && v.ld == c.ld && v.rows == c.rows && v.cols == c.cols) return (int)i;
        }
        CUtensorMap m;
        if (!make_map_f32(&m, c.p, c.rows, c.cols, c.ld, 32, 32)) return -1;
        tmaps.push_back(m);
        tmap_views.push_back(c);
        return (int)tmaps.size() - 1;
    }
    void flush_tmaps(Op& o) {
        o.ntmaps = (int)tmaps.size();
        o.tmaps_off = tmaps.empty() ? 0 : put_blob(tmaps.data(), tmaps.size() * sizeof(CUtensorMap));
        tmaps.clear();
        tmap_views.clear();
    }

    // Queue a grouped-GEMM op (its maps / refs already set) with its leaves and targets.
    void emit_grouped(Op& o, std::vector<Leaf>& leaves, std::vector<Target>& tg, int nflags) {
        if (batch && o.kind == OP_GEMM_TF32) {
            const int base = (int)bmaps.size(), tbase = (int)btargets.size();
            for (int i = 0; i < 4; ++i) bmaps.push_back(o.maps.m[i]);
            for (const Target& t : tg) btargets.push_back(t);  // target-map indices accumulate in tmaps
            for (Leaf lf : leaves) {
                lf.a_map += base;
                lf.b_map += base;
                lf.tgt_begin += tbase;
                lf.tile_begin += bitems;
                bleaves.push_back(lf);
            }
            bitems += o.items;
            return;
        }
        o.nleaves = (int)leaves.size();
        o.leaves_off = put_blob(leaves.data(), leaves.size() * sizeof(Leaf));
        o.targets_off = put_blob(tg.data(), tg.size() * sizeof(Target));
        // many leaves: a table of every item's leaf replaces the kernel's per-tile binary search
        if ((o.kind == OP_GEMM_TF32 || o.kind == OP_GEMM_BF16X3 || o.kind == OP_GEMM_TF32X3) && leaves.size() > 4 &&
            o.items > 0 && !o.has_layout) {
            const long long tm = o.pair ? 2 * tf32_tile_m() : tf32_tile_m();
            std::vector<int> il(o.items, 0);
            for (size_t i = 0; i < leaves.size(); ++i) {
                const Leaf& lf = leaves[i];
                const long long cnt = ceil_div(lf.m, tm) * lf.tiles_n;
                for (long long t = 0; t < cnt && lf.tile_begin + t < o.items; ++t) il[lf.tile_begin + t] = (int)i;
            }
            o.has_item_leaf = true;
            o.item_leaf_off = put_blob(il.data(), il.size() * sizeof(int));
        }
        flush_tmaps(o);
        if (nflags > 0) {
            std::vector<unsigned> zeros(nflags + 2, 0u);  // + the launch epoch and finished-CTA count
            o.nflags = nflags;
            o.flags_off = put_blob(zeros.data(), zeros.size() * sizeof(unsigned));
        }
        push(o);
    }

    // One leaf product c (=|+=) a b on the tensor cores (FP32: b as stored, or as B^T in bt
    // storage) or, for FP64,
    // on the SIMT kernel.
    bool gemm(View a, View b, View c, int mode) {
        if (c.rows <= 0 || c.cols <= 0) return true;
        if (a.cols == 0) {
            if (mode == TGT_STORE) memset0(c);
            return true;
        }
        if (eb == 8) {
            if (dry) return true;
            return simt(a, b, c, mode);
        }
        if (bf || x3) return gemm_split(a, b, c, mode);
        if (dry) return true;
        Target t = make_target(c, 1.f, mode, target_map(c));
        Leaf lf;
        memset(&lf, 0, sizeof(lf));
        lf.tag = -1;
        lf.a_map = 0;
        lf.b_map = 1;
        lf.m = c.rows;
        lf.n = c.cols;
        lf.tgt_begin = 0;
        lf.tgt_count = 1;
        lf.tile_begin = 0;
        Op o;
        o.kind = OP_GEMM_TF32;
        o.bn = force_bn ? force_bn : tf32_bn(c.cols);
        lf.kblocks = (int)ceil_div(a.cols, tf32_tile_k());
        lf.tiles_n = (int)ceil_div(c.cols, o.bn);
        o.nmaj = nmaj;
        if (!make_map_f32(&o.maps.m[0], a.p, a.rows, a.cols, a.ld, 32, tf32_tile_m()) ||
            !(nmaj ? make_map_f32_n(&o.maps.m[1], b.p, b.rows, b.cols, b.ld)
                   : make_map_f32(&o.maps.m[1], b.p, b.rows, b.cols, b.ld, 32, b_box(o.bn)))) {
            err = "tensor map encoding failed (alignment?)";
            return false;
        }
        o.items = (int)(ceil_div(c.rows, tf32_tile_m()) * lf.tiles_n);
        std::vector<Leaf> lv(1, lf);
        std::vector<Target> tv(1, t);
        if (pair_ok(o.bn)) to_pair(o, lv);
        emit_grouped(o, lv, tv, 0);
        return true;
    }

    // Split leaf (split-BF16 or compensated TF32): both operands split into (hi, lo) halves in
    // workspace (released once the launch is queued: later ops run after it on the same stream),
    // then one launch.
    bool gemm_split(View a, View b, View c, int mode) {
        const size_t mark = ws_top;
        View ah, al, bh, bl;
        split(a, ah, al);
        split(b, bh, bl);
        bool ok = true;
        if (!dry) {
            Target t = make_target(c, 1.f, mode, target_map(c));
            Leaf lf;
            memset(&lf, 0, sizeof(lf));
            lf.tag = -1;
            lf.a_map = 0;
            lf.b_map = 1;
            lf.m = c.rows;
            lf.n = c.cols;
            lf.tgt_count = 1;
            Op o;
            o.kind = x3 ? OP_GEMM_TF32X3 : OP_GEMM_BF16X3;
            o.bn = bn_override() ? bn_override() : (x3 || c.cols <= 128 ? 128 : 256);
            lf.kblocks = (int)ceil_div(a.cols, x3 ? tf32_tile_k() : bf16x3_tile_k());
            lf.tiles_n = (int)ceil_div(c.cols, o.bn);
            if (x3)
                ok = make_map_f32(&o.maps.m[0], ah.p, ah.rows, ah.cols, ah.ld, 32, tf32_tile_m()) &&
                     make_map_f32(&o.maps.m[1], al.p, al.rows, al.cols, al.ld, 32, tf32_tile_m()) &&
                     make_map_f32_n(&o.maps.m[2], bh.p, bh.rows, bh.cols, bh.ld) &&
                     make_map_f32_n(&o.maps.m[3], bl.p, bl.rows, bl.cols, bl.ld);
            else
                ok = make_map_bf16(&o.maps.m[0], ah.p, ah.rows, ah.cols, ah.ld, tf32_tile_m()) &&
                     make_map_bf16(&o.maps.m[1], al.p, al.rows, al.cols, al.ld, tf32_tile_m()) &&
                     make_map_bf16(&o.maps.m[2], bh.p, bh.rows, bh.cols, bh.ld, 64) &&
                     make_map_bf16(&o.maps.m[3], bl.p, bl.rows, bl.cols, bl.ld, 64);
            if (!ok) err = "split-leaf tensor map encoding failed";
            o.items = (int)(ceil_div(c.rows, tf32_tile_m()) * lf.tiles_n);
            if (!x3 && pair_ok(o.bn)) {  // 256-row tiles on CTA pairs
                o.items = (int)(ceil_div(c.rows, 2 * tf32_tile_m()) * lf.tiles_n);
                o.pair = true;
            }
            o.nleaves = 1;
            o.leaves_off = put_blob(&lf, sizeof(lf));
            o.targets_off = put_blob(&t, sizeof(t));
            flush_tmaps(o);
            push(o);
        }
        ws_top = mark;
        return ok;
    }

    // SIMT product c (=|+=) a b with b in logical orientation (k x n).
    bool simt(View a, View b, View c, int mode) {
        if (c.rows <= 0 || c.cols <= 0) return true;
        if (a.cols == 0) {
            if (mode == TGT_STORE) memset0(c);
            return true;
        }
        if (dry) return true;
        Target t = make_target(c, 1.f, mode);
        Leaf lf;
        memset(&lf, 0, sizeof(lf));
        lf.tag = -1;
        lf.a_map = 0;
        lf.b_map = 1;
        lf.m = c.rows;
        lf.n = c.cols;
        lf.kblocks = a.cols;
        lf.tiles_n = (int)ceil_div(c.cols, F64_BN);
        lf.tgt_count = 1;
        Op o;
        o.kind = OP_GEMM_SIMT;
        o.eb = eb;
        o.wtile = wtile && eb == 8;
        MatRef refs[2] = {{a.p, a.ld, a.rows, a.cols}, {b.p, b.ld, b.rows, b.cols}};
        o.refs_off = put_blob(refs, sizeof(refs));
        o.items = (int)(ceil_div(c.rows, F64_BM) * lf.tiles_n);
        o.nleaves = 1;
        o.leaves_off = put_blob(&lf, sizeof(lf));
        o.targets_off = put_blob(&t, sizeof(t));
        push(o);
        return true;
    }

    // ---------------------------------------------------------- materialised schedules
    bool product(View a, View b, View c, int L) {
        if (L == 0) return gemm(a, b, c, TGT_STORE);
        if (fused_below > 0 && L <= fused_below) {
            // the fused bottom of a deep FUSED product; its sum slots are free again once its
            // launches are queued (everything after it runs later on the same stream)
            const size_t mark = ws_top;
            const bool ok = fused(a, b, c, L);
            ws_top = mark;
            return ok;
        }
        if (sched == SW_SCHED_TWO_TEMP || (fused_below > 0 && algo == SW_ALGO_WINOGRAD)) return two_temp(a, b, c, L);
        if (sched == SW_SCHED_IN_PLACE) return in_place(a, b, c, L);
        return algo == SW_ALGO_STRASSEN ? alloc_strassen(a, b, c, L) : alloc_winograd(a, b, c, L);
    }

    // Alg. 2 (Sec. 2.2) with fresh temporaries: two operand sums, seven products.
    bool alloc_strassen(View a, View b, View c, int L) {
        View A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
        View B11 = quadB(b, 0), B12 = quadB(b, 1), B21 = quadB(b, 2), B22 = quadB(b, 3);
        View C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
        const int k2 = A11.cols;
        const size_t mark = ws_top;
        View sa = talloc(A11.rows, k2), sb = tallocB(k2, C11.cols), P[7];
        for (int i = 0; i < 7; ++i) P[i] = talloc(C11.rows, C11.cols);
        bool ok = true;
        add(sa, A11, A22, +1); add(sb, B11, B22, +1); ok &= product(sa, sb, P[0], L - 1);
        add(sa, A21, A22, +1); ok &= product(sa, B11, P[1], L - 1);
        add(sb, B12, B22, -1); ok &= product(A11, sb, P[2], L - 1);
        add(sb, B21, B11, -1); ok &= product(A22, sb, P[3], L - 1);
        add(sa, A11, A12, +1); ok &= product(sa, B22, P[4], L - 1);
        add(sa, A21, A11, -1); add(sb, B11, B12, +1); ok &= product(sa, sb, P[5], L - 1);
        add(sa, A12, A22, -1); add(sb, B21, B22, +1); ok &= product(sa, sb, P[6], L - 1);
        // C11 = P1 + P4 - P5 + P7 ; C12 = P3 + P5 ; C21 = P2 + P4 ; C22 = P1 + P3 - P2 + P6
        add(C11, P[0], P[3], +1); add(C11, C11, P[4], -1); add(C11, C11, P[6], +1);
        add(C12, P[2], P[4], +1);
        add(C21, P[1], P[3], +1);
        add(C22, P[0], P[2], +1); add(C22, C22, P[1], -1); add(C22, C22, P[5], +1);
        ws_top = mark;
        return ok;
    }

    // Alg. 3 with the BDPZ 22-operation form (Sec. 2.3): 4 S, 4 T and 7 P temporaries per
    // level; the U chain reuses the P blocks once they are consumed.
    bool alloc_winograd(View a, View b, View c, int L) {
        View A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
        View B11 = quadB(b, 0), B12 = quadB(b, 1), B21 = quadB(b, 2), B22 = quadB(b, 3);
        View C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
        const int m2 = A11.rows, k2 = A11.cols, n2 = C11.cols;
        const size_t mark = ws_top;
        View S1 = talloc(m2, k2), S2 = talloc(m2, k2), S3 = talloc(m2, k2), S4 = talloc(m2, k2);
        View T1 = tallocB(k2, n2), T2 = tallocB(k2, n2), T3 = tallocB(k2, n2), T4 = tallocB(k2, n2);
        View P[7];
        for (int i = 0; i < 7; ++i) P[i] = talloc(m2, n2);
        bool ok = true;
        add(S1, A21, A22, +1);
        add(S2, S1, A11, -1);
        add(S3, A11, A21, -1);
        add(T1, B12, B11, -1);
        add(T2, B22, T1, -1);
        add(T3, B22, B12, -1);
        add(S4, A12, S2, -1);
        add(T4, T2, B21, -1);
        ok &= product(A11, B11, P[0], L - 1);
        ok &= product(A12, B21, P[1], L - 1);
        ok &= product(S4, B22, P[2], L - 1);
        ok &= product(A22, T4, P[3], L - 1);
        ok &= product(S1, T1, P[4], L - 1);
        ok &= product(S2, T2, P[5], L - 1);
        ok &= product(S3, T3, P[6], L - 1);
        add(C11, P[0], P[1], +1);  // U1 = P1 + P2
        add(P[5], P[0], P[5], +1); // U2 = P1 + P6
        add(P[6], P[5], P[6], +1); // U3 = U2 + P7
        add(P[0], P[5], P[4], +1); // U4 = U2 + P5
        add(C12, P[0], P[2], +1);  // U5 = U4 + P3
        add(C21, P[6], P[3], -1);  // U6 = U3 - P4
        add(C22, P[6], P[4], +1);  // U7 = U3 + P5
        ws_top = mark;
        return ok;
    }

    // Table 2 (Sec. 3.3): two temporaries per level, X (A-quadrant sums, then P1) and Y.
    bool two_temp(View a, View b, View c, int L) {
        View A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
        View B11 = quadB(b, 0), B12 = quadB(b, 1), B21 = quadB(b, 2), B22 = quadB(b, 3);
        View C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
        const int m2 = A11.rows, k2 = A11.cols, n2 = C11.cols;
        const size_t mark = ws_top;
        View X = talloc(m2, std::max(k2, n2));
        View Xp = X;                           // X as P1 (m2 x n2)
        Xp.cols = n2;
        Xp.ld = round_up(std::max(n2, 1), 4);
        X.cols = k2;                           // X as an A-quadrant sum (m2 x k2)
        X.ld = round_up(std::max(k2, 1), 4);
        View Y = tallocB(k2, n2);
        bool ok = true;
        add(X, A11, A21, -1);                  //  1  S3 = A11 - A21      -> X
        add(Y, B22, B12, -1);                  //  2  T3 = B22 - B12      -> Y
        ok &= product(X, Y, C21, L - 1);       //  3  P7 = S3 T3          -> C21
        add(X, A21, A22, +1);                  //  4  S1 = A21 + A22      -> X
        add(Y, B12, B11, -1);                  //  5  T1 = B12 - B11      -> Y
        ok &= product(X, Y, C22, L - 1);       //  6  P5 = S1 T1          -> C22
        add(X, X, A11, -1);                    //  7  S2 = S1 - A11       -> X
        add(Y, B22, Y, -1);                    //  8  T2 = B22 - T1       -> Y
        ok &= product(X, Y, C12, L - 1);       //  9  P6 = S2 T2          -> C12
        add(X, A12, X, -1);                    // 10  S4 = A12 - S2       -> X
        ok &= product(X, B22, C11, L - 1);     // 11  P3 = S4 B22         -> C11
        ok &= product(A11, B11, Xp, L - 1);    // 12  P1 = A11 B11        -> X
        add(C12, Xp, C12, +1);                 // 13  U2 = P1 + P6        -> C12
        add(C21, C12, C21, +1);                // 14  U3 = U2 + P7        -> C21
        add(C12, C12, C22, +1);                // 15  U4 = U2 + P5        -> C12
        add(C22, C21, C22, +1);                // 16  U7 = U3 + P5        -> C22
        add(C12, C12, C11, +1);                // 17  U5 = U4 + P3        -> C12
        add(Y, Y, B21, -1);                    // 18  T4 = T2 - B21       -> Y
        ok &= product(A22, Y, C11, L - 1);     // 19  P4 = A22 T4         -> C11
        add(C21, C21, C11, -1);                // 20  U6 = U3 - P4        -> C21
        ok &= product(A12, B21, C11, L - 1);   // 21  P2 = A12 B21        -> C11
        add(C11, Xp, C11, +1);                 // 22  U1 = P1 + P2        -> C11
        ws_top = mark;
        return ok;
    }

    // Table 3 (Sec. 3.3): temporaries stored in the quadrants of A, B and C.  Sub-products
    // recurse in place too, so each one may overwrite its two operand blocks; the table's
    // order never reads a block after such a product consumed it.  Square only: the C22
    // quadrant holds the B-side values T1 and T4 (held transposed like every B-side value).
    bool in_place(View a, View b, View c, int L) {
        View A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
        View B11 = quadB(b, 0), B12 = quadB(b, 1), B21 = quadB(b, 2), B22 = quadB(b, 3);
        View C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
        bool ok = true;
        add(C11, A11, A21, -1);                //  1  S3 = A11 - A21      -> C11
        add(A21, A21, A22, +1);                //  2  S1 = A21 + A22      -> A21
        add(C22, B12, B11, -1);                //  3  T1 = B12 - B11      -> C22
        add(B12, B22, B12, -1);                //  4  T3 = B22 - B12      -> B12
        ok &= product(C11, B12, C21, L - 1);   //  5  P7 = S3 T3          -> C21
        add(C12, A21, A11, -1);                //  6  S2 = S1 - A11       -> C12
        ok &= product(A11, B11, C11, L - 1);   //  7  P1 = A11 B11        -> C11
        add(B11, B22, C22, -1);                //  8  T2 = B22 - T1       -> B11
        ok &= product(A21, C22, A11, L - 1);   //  9  P5 = S1 T1          -> A11
        add(C22, B11, B21, -1);                // 10  T4 = T2 - B21       -> C22
        ok &= product(A22, C22, A21, L - 1);   // 11  P4 = A22 T4         -> A21
        add(A22, A12, C12, -1);                // 12  S4 = A12 - S2       -> A22
        ok &= product(C12, B11, C22, L - 1);   // 13  P6 = S2 T2          -> C22
        add(C22, C11, C22, +1);                // 14  U2 = P1 + P6        -> C22
        ok &= product(A12, B21, C12, L - 1);   // 15  P2 = A12 B21        -> C12
        add(C11, C11, C12, +1);                // 16  U1 = P1 + P2        -> C11
        add(C12, C22, A11, +1);                // 17  U4 = U2 + P5        -> C12
        add(C22, C22, C21, +1);                // 18  U3 = U2 + P7        -> C22
        add(C21, C22, A21, -1);                // 19  U6 = U3 - P4        -> C21
        add(C22, C22, A11, +1);                // 20  U7 = U3 + P5        -> C22
        ok &= product(A22, B22, A12, L - 1);   // 21  P3 = S4 B22         -> A12
        add(C12, C12, A12, +1);                // 22  U5 = U4 + P3        -> C12
        return ok;
    }

    // ---------------------------------------------------------- FUSED
    // Per-level coefficient tables of the 7 products.
    struct Term { int q; int s; };  // quadrant (0:11 1:12 2:21 3:22), sign
    struct ProdTab {
        int pure_a_q[7];  // quadrant of A if the A operand is a single block, else -1
        int pure_b_q[7];
        int ntgt[7];
        Term tgt[7][4];
    };

    static const ProdTab& table(int algo) {
        // Winograd, BDPZ (Sec. 2.3): C11 = U1 = P1+P2, C12 = U5 = P1+P6+P5+P3,
        // C21 = U6 = P1+P6+P7-P4, C22 = U7 = P1+P6+P7+P5.
        static const ProdTab win = {
            {0, 1, -1, 3, -1, -1, -1},
            {0, 2, 3, -1, -1, -1, -1},
            {4, 1, 1, 1, 2, 3, 2},
            {{{0, 1}, {1, 1}, {2, 1}, {3, 1}},
             {{0, 1}},
             {{1, 1}},
             {{2, -1}},
             {{1, 1}, {3, 1}},
             {{1, 1}, {2, 1}, {3, 1}},
             {{2, 1}, {3, 1}}}};
        // Strassen (Sec. 2.2): C11 = P1+P4-P5+P7, C12 = P3+P5, C21 = P2+P4, C22 = P1+P3-P2+P6.
        static const ProdTab str = {
            {-1, -1, 0, 3, -1, -1, -1},
            {-1, 0, -1, -1, 3, -1, -1},
            {2, 2, 2, 2, 2, 1, 1},
            {{{0, 1}, {3, 1}},
             {{2, 1}, {3, -1}},
             {{1, 1}, {3, 1}},
             {{0, 1}, {2, 1}},
             {{0, -1}, {1, 1}},
             {{3, 1}},
             {{0, 1}}}};
        // Winograd in Knuth's form (Sec. 2.3), a, b, c, d = A11, A12, A21, A22 and A, C, B, D =
        // B11, B12, B21, B22: products aA, bB, (a+b-c-d)D, d(B+C-A-D), v = (c+d)(C-A),
        // (c+d-a)(A+D-C) (w = aA + this), u = (c-a)(C-D); C11 = aA+bB, C12 = w+v+(a+b-c-d)D,
        // C21 = w+u+d(B+C-A-D), C22 = w+u+v.  The same seven products as BDPZ up to the sign of the
        // fourth; its operand sums are grouped as Knuth writes them.
        static const ProdTab knuth = {
            {0, 1, -1, 3, -1, -1, -1},
            {0, 2, 3, -1, -1, -1, -1},
            {4, 1, 1, 1, 2, 3, 2},
            {{{0, 1}, {1, 1}, {2, 1}, {3, 1}},
             {{0, 1}},
             {{1, 1}},
             {{2, 1}},
             {{1, 1}, {3, 1}},
             {{1, 1}, {2, 1}, {3, 1}},
             {{2, 1}, {3, 1}}}};
        return algo == SW_ALGO_STRASSEN ? str : algo == SW_ALGO_WINOGRAD_KNUTH ? knuth : win;
    }

    // ---------------------------------------------------------- accumulation chains (depth 1)
    // One Winograd level (BDPZ or Knuth's grouping; the same product structure) with the sums
    // kept in tensor memory: a CTA pair's tile that continues the accumulator of its tile two
    // items back adds the next product to the running sum, so C receives
    //   [P1 -> C11 := ; +P6 -> C12 := U2 ; +P7 -> C21 := C22 := U3]  (stores, the first writers)
    //   [P5 -> C22 += ; +P3 -> C12 += P5 + P3]   [P2 -> C11 +=]   [P4 -> C21 += sign P4]
    // (4 stores and 4 reduce-adds instead of 4 and 10).  The work layout is explicit: every CTA
    // pair gets its own item sequence (pairs of positions, so the two accumulators alternate, or
    // single positions with the one accumulator of 512-wide tiles; stores before adds on every
    // pair; greedy balance), interleaved as item t * units + u.
    // *done = 1 when the op was emitted; 0 to fall back to the plain FUSED order.
    // `o` is the depth-1 grouped-GEMM op with its kind, tile width and operand maps set (TF32 on
    // CTA pairs, or split-BF16 on single CTAs).
    bool chain_plan(const ProdTab& T, Op o, View C, const std::vector<Leaf>& base, int mb, int nb, int bn,
                    const std::vector<int>& flag_base, const std::vector<int>& flag_cols, int nflags, int* done) {
        static const bool off = getenv("SWMM_NO_CHAINS") != nullptr;  // diagnostics
        *done = 0;
        if (off || dry) return true;
        const bool pairs = o.pair;
        const int units = !pairs ? sms  // one CTA per SM, all resident
                                 : o.kind == OP_GEMM_TF32 ? gemm_tf32n_pair_units(sms, bn) : gemm_bf16x3_pair_units(sms);
        const int nacc = bn > 256 ? 1 : 2;  // TMEM accumulators: a chain's next step comes nacc items later
        const int tile_m = pairs ? 2 * tf32_tile_m() : tf32_tile_m();
        if (units <= 0) return true;
        struct Emit { int q, mode; float sign; };
        struct Chain { int len; int prod[3]; int nemit[3]; Emit emit[3][2]; };
        const float s4 = T.ntgt[3] == 1 && T.tgt[3][0].q == 2 ? (float)T.tgt[3][0].s : 0.f;
        const Chain chains[4] = {
            {3, {0, 5, 6}, {1, 1, 2},
             {{{0, TGT_STORE, 1.f}}, {{1, TGT_STORE, 1.f}}, {{2, TGT_STORE, 1.f}, {3, TGT_STORE, 1.f}}}},
            {2, {4, 2, 0}, {1, 1, 0}, {{{3, TGT_ATOMIC, 1.f}}, {{1, TGT_ATOMIC, 1.f}}}},
            {1, {1, 0, 0}, {1, 0, 0}, {{{0, TGT_ATOMIC, 1.f}}}},
            {1, {3, 0, 0}, {1, 0, 0}, {{{2, TGT_ATOMIC, s4}}}}};
        // the chains must add up to the product table's combination, else keep the plain order
        float coef[7][4] = {}, want[7][4] = {};
        for (int p = 0; p < 7; ++p)
            for (int t = 0; t < T.ntgt[p]; ++t) want[p][T.tgt[p][t].q] += (float)T.tgt[p][t].s;
        for (const Chain& ch : chains)
            for (int st = 0; st < ch.len; ++st)
                for (int e = 0; e < ch.nemit[st]; ++e)
                    for (int j = 0; j <= st; ++j) coef[ch.prod[j]][ch.emit[st][e].q] += ch.emit[st][e].sign;
        for (int p = 0; p < 7; ++p)
            for (int q = 0; q < 4; ++q)
                if (coef[p][q] != want[p][q]) return true;
        // leaves: one per product (whole quadrant) with its chain step's targets, plus a no-op leaf
        std::vector<Leaf> leaves(8);
        std::vector<Target> tg;
        for (const Chain& ch : chains)
            for (int st = 0; st < ch.len; ++st) {
                Leaf lf = base[ch.prod[st]];
                lf.c_row0 = lf.c_col0 = 0;
                lf.cont = st > 0 ? 1 : 0;
                lf.tgt_begin = (int)tg.size();
                for (int e = 0; e < ch.nemit[st]; ++e) {
                    const Emit& em = ch.emit[st][e];
                    const int r = em.q >> 1, c = em.q & 1;
                    View cv = sub(C, (long long)r * mb, (long long)c * nb, std::min(mb, C.rows - r * mb),
                                  std::min(nb, C.cols - c * nb), eb);
                    if (cv.rows <= 0 || cv.cols <= 0) continue;
                    Target t = make_target(cv, em.sign, em.mode, target_map(cv));
                    t.flag_base = flag_base[em.q];
                    t.flag_cols = flag_cols[em.q];
                    tg.push_back(t);
                }
                lf.tgt_count = (int)tg.size() - lf.tgt_begin;
                leaves[ch.prod[st]] = lf;
            }
        Leaf& nop = leaves[7];
        memset(&nop, 0, sizeof(nop));
        nop.tag = -1;
        nop.a_map = 0;
        nop.b_map = 1;
        nop.tiles_n = 1;
        // positions: tiles of a quadrant, in groups of GR tile rows, column-major in a group;
        // GR ~ sqrt(2 units) makes the tiles one wave of pair jobs covers about square, so the A
        // and B blocks they read are shared by as many tiles as possible
        const int tm2 = (int)ceil_div(mb, tile_m), tn = (int)ceil_div(nb, bn);
        const int GR = std::max(1, (int)std::lround(std::sqrt(2.0 * units)));
        std::vector<int> pos;
        for (int g0 = 0; g0 < tm2; g0 += GR)
            for (int c = 0; c < tn; ++c)
                for (int r = g0; r < std::min(tm2, g0 + GR); ++r) pos.push_back(r << 16 | c);
        const int npos = (int)pos.size();
        // jobs in order: chain pairs (chains A, B), then single products; each to the least loaded unit
        std::vector<std::vector<std::pair<int, int>>> seq(units);  // (leaf, tile) per unit
        std::vector<int> load(units, 0);
        auto least = [&]() {
            int u = 0;
            for (int i = 1; i < units; ++i)
                if (load[i] < load[u]) u = i;
            return u;
        };
        for (const Chain& ch : chains) {
            if (ch.len == 1) {
                for (int p = 0; p < npos; ++p) {
                    const int u = least();
                    seq[u].push_back({ch.prod[0], pos[p]});
                    load[u] += 1;
                }
                continue;
            }
            for (int p = 0; p < npos; p += nacc) {
                const int u = least();
                for (int st = 0; st < ch.len; ++st) {
                    seq[u].push_back({ch.prod[st], pos[p]});
                    if (nacc == 2)
                        seq[u].push_back(p + 1 < npos ? std::make_pair(ch.prod[st], pos[p + 1]) : std::make_pair(7, 0));
                }
                load[u] += ch.len * (nacc == 2 && p + 1 < npos ? 2 : 1);
            }
        }
        size_t tmax = 0;
        for (const auto& q : seq) tmax = std::max(tmax, q.size());
        std::vector<int> il(tmax * units, 7), it(tmax * units, 0);
        for (int u = 0; u < units; ++u)
            for (size_t t = 0; t < seq[u].size(); ++t) {
                il[t * units + u] = seq[u][t].first;
                it[t * units + u] = seq[u][t].second;
            }
        o.items = (int)(tmax * units);
        o.units = units;
        o.has_layout = true;
        o.item_leaf_off = put_blob(il.data(), il.size() * sizeof(int));
        o.item_tile_off = put_blob(it.data(), it.size() * sizeof(int));
        emit_grouped(o, leaves, tg, nflags);
        *done = 1;
        return true;
    }
    // FUSED plan for C (m x n) <- A (m x k) B (k x n) at depth L (1..3).  `B` is in bt storage
    // on the FP32 path (B^T, n x k).
    bool fused(View A, View B, View C, int L) {
        const ProdTab& T = table(algo);
        const int m = C.rows, n = C.cols, k = A.cols;
        const int s = 1 << L;
        const int mb = (int)ceil_div(m, s);
        const int kb = eb == 8 ? (int)ceil_div(k, s)
                               : (int)round_up(ceil_div(k, s), bf ? bf16x3_tile_k() : tf32_tile_k());
        const int nb = eb == 8 ? (int)ceil_div(n, s) : (int)round_up(ceil_div(n, s), bf ? 8 : 4);
        int nleaf = 1;
        for (int i = 0; i < L; ++i) nleaf *= 7;
        std::vector<short> slot_a(nleaf, -1), slot_b(nleaf, -1);
        std::vector<int> ar(nleaf), ac(nleaf), br(nleaf), bc(nleaf);
        int na = 0, nbs = 0;
        for (int w = 0; w < nleaf; ++w) {
            bool pa = true, pb = true;
            int r_a = 0, c_a = 0, r_b = 0, c_b = 0;
            for (int l = 0, div = nleaf / 7; l < L; ++l, div /= 7) {
                const int p = (w / div) % 7;
                const int qa = T.pure_a_q[p], qb = T.pure_b_q[p];
                if (qa < 0) pa = false;
                if (qb < 0) pb = false;
                r_a = r_a * 2 + (qa >= 0 ? (qa >> 1) : 0);
                c_a = c_a * 2 + (qa >= 0 ? (qa & 1) : 0);
                r_b = r_b * 2 + (qb >= 0 ? (qb >> 1) : 0);
                c_b = c_b * 2 + (qb >= 0 ? (qb & 1) : 0);
            }
            if (pa) { ar[w] = r_a * mb; ac[w] = c_a * kb; } else { slot_a[w] = (short)na++; }
            if (pb) {  // logical block (r_b, c_b) of B; in bt storage it is block (c_b, r_b) of B^T
                if (bt) { br[w] = c_b * nb; bc[w] = r_b * kb; } else { br[w] = r_b * kb; bc[w] = c_b * nb; }
            } else {
                slot_b[w] = (short)nbs++;
            }
        }
        // Split-BF16 leaves at depth 1 or 2 with A and B read as stored: one pass per side writes the
        // bf16 halves of the operand and of its sums (no FP32 sum slots, no separate split passes)
        const bool split_sums = bf && !x3 && L <= 2 && na > 0 && nbs > 0 && !bt && vec_ok(A) && vec_ok(B) &&
                                (kb % 8) == 0 && (nb % 8) == 0;
        // scratch for the materialised operand sums: dense slots, row stride = block width
        View SA = split_sums ? View{nullptr, kb, na * mb, kb} : talloc(std::max(na, 1) * mb, kb);
        SA.rows = na * mb;
        SA.ld = kb;
        View SB = split_sums ? View{nullptr, nb, nbs * kb, nb}
                             : bt ? talloc(std::max(nbs, 1) * nb, kb) : talloc(std::max(nbs, 1) * kb, nb);
        SB.rows = bt ? nbs * nb : nbs * kb;
        SB.ld = bt ? kb : nb;
        // split-BF16 leaves: (hi, lo) halves of A, B and the S / T sums (sized in the dry run too)
        View halves[4][2];
        if (bf || x3) {
            const int hr[4] = {m, k, std::max(SA.rows, 1), std::max(SB.rows, 1)};
            const int hc[4] = {k, n, kb, nb};
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 2; ++j) halves[i][j] = talloc_half(hr[i], hc[i]);
        }
        if (dry) return true;
        // operand-sum passes over A and over B (FP32: one launch for both sides; split-BF16: the
        // halves of A, B and their sums in one pass per side)
        Op pa, pb;
        if (na > 0) {
            pa.kind = OP_PREADD;
            pa.eb = eb;
            PreaddArgs& p = pa.pre;
            memset(&p, 0, sizeof(p));
            p.x = A.p; p.ldx = A.ld; p.rows = m; p.cols = k; p.brows = mb; p.bcols = kb;
            p.out = SA.p; p.L = L; p.alg = algo == SW_ALGO_STRASSEN ? 1 : algo == SW_ALGO_WINOGRAD_KNUTH ? 3 : 2; p.bside = 0; p.bt = 0;
            for (int w = 0; w < 343; ++w) p.slot_of[w] = w < nleaf ? slot_a[w] : (short)-1;
        }
        if (nbs > 0) {
            pb.kind = OP_PREADD;
            pb.eb = eb;
            PreaddArgs& p = pb.pre;
            memset(&p, 0, sizeof(p));
            p.x = B.p; p.ldx = B.ld;
            if (bt) { p.rows = n; p.cols = k; p.brows = nb; p.bcols = kb; }
            else { p.rows = k; p.cols = n; p.brows = kb; p.bcols = nb; }
            p.out = SB.p; p.L = L; p.alg = algo == SW_ALGO_STRASSEN ? 1 : algo == SW_ALGO_WINOGRAD_KNUTH ? 3 : 2; p.bside = 1; p.bt = bt ? 1 : 0;
            for (int w = 0; w < 343; ++w) p.slot_of[w] = w < nleaf ? slot_b[w] : (short)-1;
        }
        if (split_sums) {
            pa.kind = OP_PREADD_SPLIT;
            pa.sout = {reinterpret_cast<__nv_bfloat16*>(halves[0][0].p), reinterpret_cast<__nv_bfloat16*>(halves[0][1].p),
                       halves[0][0].ld, reinterpret_cast<__nv_bfloat16*>(halves[2][0].p),
                       reinterpret_cast<__nv_bfloat16*>(halves[2][1].p)};
            pb.sout = {reinterpret_cast<__nv_bfloat16*>(halves[1][0].p), reinterpret_cast<__nv_bfloat16*>(halves[1][1].p),
                       halves[1][0].ld, reinterpret_cast<__nv_bfloat16*>(halves[3][0].p),
                       reinterpret_cast<__nv_bfloat16*>(halves[3][1].p)};
            pa.pre_b = pb.pre;
            pa.sout_b = pb.sout;
            push(pa);
        } else if (na > 0 && nbs > 0 && eb == 4) {
            pa.pre_b = pb.pre;
            pa.pre_two = true;
            push(pa);
        } else {
            if (na > 0) push(pa);
            if (nbs > 0) push(pb);
        }
        // Each C block's first writer (the first leaf, in leaf order, that adds into it) stores
        // instead of adding; later leaves wait for it tile by tile.  Used at depth 1 on the TF32
        // path, where the first writer's tiles lead their position group and the waits are short;
        // deeper levels (many leaves queue behind one writer) and the SIMT FP64 leaf keep a zeroed
        // C and reduce-adds only.
        const bool ordered = eb == 4 && L == 1 && !batch && !server;
        if (!ordered) memset0(C);
        const int bn_o = eb == 8                ? F64_BN
                         : force_bn             ? force_bn
                         : x3 || (bf && nb <= 128) ? 128
                         : bf                   ? 256
                                                : tf32_bn(nb);
        std::vector<int> first_writer(1 << (2 * L), -1), flag_base(1 << (2 * L), -1), flag_cols(1 << (2 * L), 0);
        int nflags = 0;
        // leaves and their Kronecker-product targets
        std::vector<Leaf> base_leaves;
        std::vector<Target> tg;
        const int tm_sz = eb == 4 ? tf32_tile_m() : F64_BM;
        const int bn = bn_o;
        for (int w = 0; w < nleaf; ++w) {
            Leaf lf;
            memset(&lf, 0, sizeof(lf));
            lf.tag = -1;
            if (slot_a[w] < 0) { lf.a_map = 0; lf.a_row = ar[w]; lf.a_col = ac[w]; }
            else { lf.a_map = 2; lf.a_row = slot_a[w] * mb; lf.a_col = 0; }
            if (slot_b[w] < 0) { lf.b_map = 1; lf.b_row = br[w]; lf.b_col = bc[w]; }
            else { lf.b_map = 3; lf.b_row = slot_b[w] * (bt ? nb : kb); lf.b_col = 0; }
            lf.m = mb;
            lf.n = nb;
            lf.kblocks = eb == 8 ? kb : kb / (bf ? bf16x3_tile_k() : tf32_tile_k());
            lf.tiles_n = (int)ceil_div(nb, bn);
            lf.tgt_begin = (int)tg.size();
            int digits[3] = {0, 0, 0};
            for (int l = 0, div = nleaf / 7; l < L; ++l, div /= 7) digits[l] = (w / div) % 7;
            int idx[3] = {0, 0, 0};
            for (;;) {
                int r = 0, c = 0;
                float sg = 1.f;
                for (int l = 0; l < L; ++l) {
                    const Term t = T.tgt[digits[l]][idx[l]];
                    r = r * 2 + (t.q >> 1);
                    c = c * 2 + (t.q & 1);
                    sg *= (float)t.s;
                }
                View cv = sub(C, (long long)r * mb, (long long)c * nb, std::min(mb, m - r * mb),
                              std::min(nb, n - c * nb), eb);
                if (cv.rows > 0 && cv.cols > 0) {
                    Target t = make_target(cv, sg, TGT_ATOMIC, target_map(cv));
                    if (ordered) {
                        const int blk = r * (1 << L) + c;
                        if (first_writer[blk] < 0) {
                            first_writer[blk] = w;
                            flag_cols[blk] = (int)ceil_div(cv.cols, bn_o);
                            flag_base[blk] = nflags;
                            nflags += (int)ceil_div(cv.rows, tm_sz) * flag_cols[blk];
                        }
                        t.mode = first_writer[blk] == w ? TGT_STORE : TGT_ATOMIC;
                        t.flag_base = flag_base[blk];
                        t.flag_cols = flag_cols[blk];
                    }
                    tg.push_back(t);
                }
                int l = L - 1;
                while (l >= 0 && ++idx[l] == T.ntgt[digits[l]]) { idx[l] = 0; --l; }
                if (l < 0) break;
            }
            lf.tgt_count = (int)tg.size() - lf.tgt_begin;
            base_leaves.push_back(lf);
        }
        // Work order: position groups of GM x GN tiles, then leaves, then tiles in the group, so
        // the C tiles every leaf of a group adds into stay in L2 while the group is processed.
        std::vector<Leaf> leaves;
        int items = 0;
        const int tiles_m = (int)ceil_div(mb, tm_sz), tiles_n = (int)ceil_div(nb, bn);
        // group shapes from a sweep at n = 8192 (depth 1: 16 x 8 tiles; depth 2: 4 x 4; depth 3: 2 x 2)
        int GM = eb == 8 ? tiles_m : (L == 1 ? 16 : L == 2 ? 4 : 2);
        int GN = eb == 8 ? tiles_n : (L == 1 ? 8 : L == 2 ? 4 : 2);
        if (const char* g = getenv("SWMM_GROUP")) {  // tuning override "GMxGN"
            int gm_ = 0, gn_ = 0;
            if (sscanf(g, "%dx%d", &gm_, &gn_) == 2 && gm_ > 0 && gn_ > 0 && eb == 4) { GM = gm_; GN = gn_; }
        }
        // CTA pairs: a group must hold whole 256-row tiles, or a pair's second half would also
        // compute rows of the next group
        if (eb == 4 && pair_ok(bn) && (GM & 1)) ++GM;
        for (int gm = 0; gm < tiles_m; gm += GM)
            for (int gn = 0; gn < tiles_n; gn += GN)
                for (const Leaf& b0 : base_leaves) {
                    Leaf lf = b0;
                    const int r0 = gm * tm_sz, c0 = gn * bn;
                    lf.m = std::min(GM * tm_sz, mb - r0);
                    lf.n = std::min(GN * bn, nb - c0);
                    lf.a_row += r0;
                    if (bt) lf.b_row += c0;  // B^T: rows are N
                    else lf.b_col += c0;
                    lf.c_row0 = r0;
                    lf.c_col0 = c0;
                    lf.tiles_n = (int)ceil_div(lf.n, bn);
                    lf.tile_begin = items;
                    items += (int)ceil_div(lf.m, tm_sz) * lf.tiles_n;
                    leaves.push_back(lf);
                }
        Op o;
        o.items = items;
        if (bf || x3) {
            // split every operand source once: A, B, and the S / T sums
            o.kind = x3 ? OP_GEMM_TF32X3 : OP_GEMM_BF16X3;
            o.bn = bn;
            View srcs[4] = {A, B, SA, SB};
            srcs[0].rows = m; srcs[0].cols = k;
            srcs[1].rows = k; srcs[1].cols = n;
            srcs[2].cols = kb;
            srcs[3].cols = nb;
            const int box[4] = {tf32_tile_m(), 64, tf32_tile_m(), 64};
            for (int i = 0; i < 4; ++i) {
                const View& hi = halves[i][0];
                const View& lo = halves[i][1];
                if (srcs[i].rows > 0 && !split_sums) split_into(srcs[i], hi, lo);
                bool mok;
                if (x3)  // A side K-major, B side N-major (i odd: B and the T sums)
                    mok = (i & 1) ? make_map_f32_n(&o.maps.m[2 * i], hi.p, hi.rows, hi.cols, hi.ld) &&
                                        make_map_f32_n(&o.maps.m[2 * i + 1], lo.p, lo.rows, lo.cols, lo.ld)
                                  : make_map_f32(&o.maps.m[2 * i], hi.p, hi.rows, hi.cols, hi.ld, 32, tf32_tile_m()) &&
                                        make_map_f32(&o.maps.m[2 * i + 1], lo.p, lo.rows, lo.cols, lo.ld, 32,
                                                     tf32_tile_m());
                else
                    mok = make_map_bf16(&o.maps.m[2 * i], hi.p, hi.rows, hi.cols, hi.ld, box[i]) &&
                          make_map_bf16(&o.maps.m[2 * i + 1], lo.p, lo.rows, lo.cols, lo.ld, box[i]);
                if (!mok) {
                    err = "split-leaf tensor map encoding failed";
                    return false;
                }
            }
            if (!x3 && pair_ok(bn)) to_pair(o, leaves);
        } else if (eb == 4) {
            o.kind = OP_GEMM_TF32;
            o.bn = bn;
            o.nmaj = nmaj;
            const bool mok =
                nmaj ? make_map_f32_n(&o.maps.m[1], B.p, k, n, B.ld) &&
                           make_map_f32_n(&o.maps.m[3], SB.p, std::max(SB.rows, 1), nb, SB.ld)
                     : make_map_f32(&o.maps.m[1], B.p, n, k, B.ld, 32, b_box(bn)) &&
                           make_map_f32(&o.maps.m[3], SB.p, std::max(SB.rows, 1), kb, SB.ld, 32, b_box(bn));
            if (!make_map_f32(&o.maps.m[0], A.p, m, k, A.ld, 32, tf32_tile_m()) || !mok ||
                !make_map_f32(&o.maps.m[2], SA.p, std::max(SA.rows, 1), kb, SA.ld, 32, tf32_tile_m())) {
                err = "tensor map encoding failed";
                return false;
            }
            if (pair_ok(bn)) to_pair(o, leaves);
        } else {
            o.kind = OP_GEMM_SIMT;
            o.eb = 8;
            o.wtile = wtile;
            MatRef refs[4] = {{A.p, A.ld, m, k}, {B.p, B.ld, k, n}, {SA.p, SA.ld, SA.rows, kb},
                              {SB.p, SB.ld, SB.rows, nb}};
            o.refs_off = put_blob(refs, sizeof(refs));
        }
        // depth-1 accumulation chains: TF32 on CTA pairs, split-BF16 on single CTAs
        if (ordered && L == 1 && (algo == SW_ALGO_WINOGRAD || algo == SW_ALGO_WINOGRAD_KNUTH) &&
            ((o.kind == OP_GEMM_TF32 && o.nmaj && o.pair) || o.kind == OP_GEMM_BF16X3)) {
            int done_ = 0;
            if (!chain_plan(T, o, C, base_leaves, mb, nb, bn, flag_base, flag_cols, nflags, &done_)) return false;
            if (done_) return true;
        }
        emit_grouped(o, leaves, tg, nflags);
        return true;
    }

    // ---------------------------------------------------------- batched (TF32 leaves)
    // Many independent products in one grouped launch: one batched copy launch packs the A and B
    // operands whose rows are not 16-byte aligned (bt storage: a batched transpose launch writes
    // every B^T instead), the depth >= 1 products add their operand-sum passes, and all leaves of
    // all products go into a single persistent GEMM launch (longest k first).  C needs no
    // staging: unaligned or ragged C blocks take the per-thread epilogue.
    bool batched(const sw_problem* probs, int count, const std::vector<int>& depth) {
        batch = true;
        force_bn = batch_bn == 128 ? 128 : 256;
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].k > probs[y].k; });
        std::vector<CopyJob> packs, trans;
        int pack_tiles = 0, trans_tiles = 0;
        std::vector<View> As(count), Bs(count), Cs(count);
        auto job = [](View src, View dst, int& tiles) {
            CopyJob j;
            j.x = src.p; j.ldx = src.ld; j.out = dst.p; j.ldo = dst.ld;
            j.src_rows = src.rows; j.src_cols = src.cols; j.out_rows = dst.rows; j.out_cols = dst.cols;
            j.tile_begin = tiles;
            j.pad_ = 0;
            tiles += (int)(ceil_div(dst.rows, BCOPY_TILE) * ceil_div(dst.cols, BCOPY_TILE));
            return j;
        };
        for (int i : order) {
            const sw_problem& q = probs[i];
            View a = {(char*)q.A, q.lda, q.m, q.k}, b = {(char*)q.B, q.ldb, q.k, q.n}, c = {(char*)q.C, q.ldc, q.m, q.n};
            if (q.m == 0 || q.n == 0 || q.k == 0) { As[i] = a; Bs[i] = b; Cs[i] = c; continue; }
            if (!vec_ok(a)) {
                View a2 = talloc(q.m, q.k);
                packs.push_back(job(a, a2, pack_tiles));
                a = a2;
            }
            if (nmaj) {  // B read as stored: packed only when its rows are not 16-byte aligned
                if (!vec_ok(b)) {
                    View b2 = talloc(q.k, q.n);
                    packs.push_back(job(b, b2, pack_tiles));
                    b = b2;
                }
            } else {
                View bt = talloc(q.n, q.k);
                trans.push_back(job(b, bt, trans_tiles));
                b = bt;
            }
            As[i] = a;
            Bs[i] = b;
            Cs[i] = c;
        }
        if (!dry) {
            for (int t = 0; t < 2; ++t) {
                std::vector<CopyJob>& jobs = t == 0 ? packs : trans;
                if (jobs.empty()) continue;
                Op o;
                o.kind = OP_BATCH_COPY;
                o.njobs = (int)jobs.size();
                o.tiles = t == 0 ? pack_tiles : trans_tiles;
                o.transpose = t;
                o.jobs_off = put_blob(jobs.data(), jobs.size() * sizeof(CopyJob));
                push(o);
            }
        }
        for (int i : order) {
            const sw_problem& q = probs[i];
            if (q.m == 0 || q.n == 0) continue;
            View c = Cs[i];
            if (q.k == 0) { memset0(c); continue; }
            const bool ok = depth[i] == 0 ? gemm(As[i], Bs[i], c, TGT_STORE) : fused(As[i], Bs[i], c, depth[i]);
            if (!ok) return false;
        }
        if (dry || bleaves.empty()) return true;
        Op o;
        o.kind = OP_GEMM_TF32;
        o.nmaj = nmaj;
        o.bn = force_bn;
        o.items = bitems;
        o.ngmaps = (int)bmaps.size();
        o.gmaps_off = put_blob(bmaps.data(), bmaps.size() * sizeof(CUtensorMap));
        if (batch_pair && nmaj && o.bn == 256) to_pair(o, bleaves);  // B maps do not depend on the width
        batch = false;  // the combined op itself is emitted normally
        emit_grouped(o, bleaves, btargets, 0);
        return true;
    }
};

}  // namespace

// ====================================================================== handle
struct Server;

struct sw_handle_s {
    Server* server = nullptr;  // the serving loop, when started
    int device = 0;
    int sms = 148;
    size_t budget = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    int* d_err = nullptr;
    unsigned long long* d_norms = nullptr;
    std::string last_error;
    std::unordered_map<std::string, Plan*> plans;
    // device buffers of the host-operand entry point
    char* io = nullptr;
    size_t io_bytes = 0;
    // profiling: event pairs around every launch while enabled
    bool prof = false;
    struct ProfRec { int kind; cudaEvent_t e0, e1; };
    std::vector<ProfRec> prof_live;
    std::vector<cudaEvent_t> prof_free;
    cudaStream_t capture_stream = nullptr;  // private stream for CUDA-graph capture
    // host-operand path: copy-in / copy-out streams and the events that order the panels
    cudaStream_t io_in = nullptr, io_out = nullptr;
    std::vector<cudaEvent_t> io_ev;
    // autotuner (cutoff <= 0): decisions per problem signature, and the last one made
    struct Tune { int cutoff = 0, bn = 0, pair = 0, candidates = 0; double ms = 0.0; };
    std::unordered_map<std::string, Tune> tuned;
    Tune last_tune;
    bool has_tune = false;
    std::mutex mu;
};

static cudaEvent_t prof_event(sw_handle h) {
    if (!h->prof_free.empty()) {
        cudaEvent_t e = h->prof_free.back();
        h->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static sw_status fail(sw_handle h, sw_status s, const std::string& msg) {
    if (h) h->last_error = msg;
    return s;
}

static sw_status cuda_fail(sw_handle h, cudaError_t e, const char* where) {
    return fail(h, SW_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static void flush_plans(sw_handle h) {
    if (h->plans.empty()) return;
    cudaDeviceSynchronize();
    for (auto& kv : h->plans) delete kv.second;
    h->plans.clear();
}

// Make the workspace at least `need` bytes (flushes cached plans, which point into it).
static sw_status ensure_ws(sw_handle h, size_t need) {
    if (need <= h->ws_bytes) return SW_OK;
    if (h->budget && need > h->budget)
        return fail(h, SW_EBUDGET, "workspace need " + std::to_string(need) + " B exceeds budget " +
                                       std::to_string(h->budget) + " B");
    flush_plans(h);
    if (h->ws) { cudaDeviceSynchronize(); cudaFree(h->ws); h->ws = nullptr; h->ws_bytes = 0; }
    size_t bytes = round_up((long long)need, 1 << 21);
    if (h->budget && bytes > h->budget) bytes = need;
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SW_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " B workspace failed");
    }
    h->ws_bytes = bytes;
    return SW_OK;
}

static int resolve_depth(int m, int n, int k, int cutoff, uint32_t variant, int eb) {
    if ((variant & SW_ALGO_MASK) == SW_ALGO_NAIVE) return 0;
    // static default where the autotuner does not run (stream capture, IN_PLACE, sw_mm_depth):
    // from the bench's sweeps, one TF32 Winograd level pays from n = 16384 on; FP64 leaves are
    // ALU-bound and gain from every level while the leaves keep >= 128 rows (the grouped FP64
    // launch then still fills the GPU with 64 x 64 tiles)
    if (cutoff <= 0) cutoff = eb == 4 ? 8192 : 128;
    int L = 0;
    while (L < 20) {
        const long long s = 1LL << L;
        const long long lo = std::min(std::min(ceil_div(m, s), ceil_div(n, s)), ceil_div(k, s));
        if (lo > cutoff) ++L; else break;
    }
    if ((variant & SW_SCHED_MASK) == SW_SCHED_FUSED) {
        // three levels fuse into one operand-sum pass and one grouped launch; FP64 Strassen /
        // BDPZ products go deeper by Alg. 2 / Table 2 steps above the fused bottom, one per
        // exact halving of m, n and k (at most three) while the fused bottom keeps a smallest side
        // of >= 1024 (smaller bottoms give their grouped launch too few tiles and spend more on
        // the bottom's FP64 reduce-adds than the level saves)
        int cap = 3;
        const uint32_t algo = variant & SW_ALGO_MASK;
        if (eb == 8 && (algo == SW_ALGO_STRASSEN || algo == SW_ALGO_WINOGRAD)) {
            const int dmin = std::min(m, std::min(n, k));
            int t = 0;
            while (t < 3 && m % (2 << t) == 0 && n % (2 << t) == 0 && k % (2 << t) == 0 && (dmin >> (t + 1)) >= 1024)
                ++t;
            cap += t;
        }
        if (L > cap) L = cap;
    }
    return L;
}

// Build the whole plan for one product (planner dry-run for sizes, then the real one).
// server: the plan's workspace starts at ws_base (a region of the serving arena), C is written
// directly (no packed copy: unaligned C blocks take the per-thread epilogue), and the leaf GEMM is
// the BN = 256 form the resident loop runs, without ordering counters.
static sw_status build_plan(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                            int m, int n, int k, int cutoff, uint32_t variant, bool dry, Plan* plan,
                            char* ws_base = nullptr, bool server = false) {
    const uint32_t algo = variant & SW_ALGO_MASK, sched = variant & SW_SCHED_MASK, odd = variant & SW_ODD_MASK;
    if (algo > SW_ALGO_WINOGRAD_KNUTH) return fail(h, SW_EINVAL, "unknown algorithm bits");
    if (sched > SW_SCHED_ALLOC) return fail(h, SW_EINVAL, "unknown schedule bits");
    if (algo == SW_ALGO_WINOGRAD_KNUTH && sched != SW_SCHED_FUSED)
        return fail(h, SW_EUNSUPPORTED, "Knuth's form runs in the FUSED schedule");
    const uint32_t leaf = variant & SW_LEAF_MASK;
    if (leaf > SW_LEAF_F64_WTILE) return fail(h, SW_EINVAL, "unknown leaf bits");
    if (leaf == SW_LEAF_F64_WTILE && eb != 8) return fail(h, SW_EINVAL, "SW_LEAF_F64_WTILE is an FP64 leaf");
    if (leaf == SW_LEAF_F64_WTILE && algo != SW_ALGO_WINOGRAD && algo != SW_ALGO_WINOGRAD_KNUTH)
        return fail(h, SW_EUNSUPPORTED, "Winograd-step leaf tiles go with the Winograd variants");
    if (algo == SW_ALGO_STRASSEN && (sched == SW_SCHED_TWO_TEMP || sched == SW_SCHED_IN_PLACE))
        return fail(h, SW_EUNSUPPORTED, "Tables 2 and 3 are Winograd schedules");
    if (sched == SW_SCHED_IN_PLACE && algo != SW_ALGO_NAIVE && !(m == n && n == k))
        return fail(h, SW_EUNSUPPORTED, "in-place schedule needs m == n == k");

    // split leaves (split-BF16 or compensated TF32): the split pass reads any layout
    const bool x3 = eb == 4 && (variant & SW_LEAF_MASK) == SW_LEAF_TF32X3;
    const bool bf_only = eb == 4 && (variant & SW_LEAF_MASK) == SW_LEAF_BF16X3;
    const bool bf = bf_only || x3;
    Planner P;
    P.eb = eb;
    P.bf = bf_only;
    P.x3 = x3;
    P.wtile = eb == 8 && leaf == SW_LEAF_F64_WTILE;
    // TF32 leaves read B N-major, as stored (no B^T staging); SWMM_TF32_BT=1 selects the B^T form
    // everywhere (diagnostics)
    P.nmaj = eb == 4 && !bf && !tf32_bt_form();
    P.bt = eb == 4 && !bf && !P.nmaj;
    P.variant = variant;
    P.dry = dry;
    P.ws_base = ws_base ? ws_base : h->ws;
    P.plan = plan;
    P.sched = (int)sched;
    P.algo = (int)algo;
    P.server = server;
    P.sms = h->sms;
    if (server && eb == 4 && !bf) P.force_bn = 256;
    const int L = resolve_depth(m, n, k, cutoff, variant, eb);
    plan->depth = L;

    View Av = {(char*)A, lda, m, k}, Bv = {(char*)B, ldb, k, n}, Cv = {(char*)C, ldc, m, n};
    // TF32 leaves read A and write C through TMA (16-byte rows); the SIMT FP64 leaf and the split
    // pass of the BF16X3 leaves read any layout, and unaligned C blocks take the per-thread epilogue
    const bool direct = L == 0 || algo == SW_ALGO_NAIVE || sched == SW_SCHED_FUSED;  // C is only a target
    const bool a_ok = eb == 8 || bf || Planner::vec_ok(Av),
               c_ok = eb == 8 || bf || (server && direct) || Planner::vec_ok(Cv);
    // B in the storage the leaves want: B itself (FP64, split-BF16, N-major TF32; copied when a
    // TMA read needs aligned rows), B^T in workspace (bt storage)
    auto stage_b = [&](View b, int rows_pad, int cols_pad) -> View {  // logical k x n -> storage
        if (!P.bt) {
            // N-major TF32 leaves read B through TMA: 16-byte aligned rows
            if (rows_pad == b.rows && cols_pad == b.cols && (!P.nmaj || Planner::vec_ok(b))) return b;
            View b2 = P.talloc(rows_pad, cols_pad);
            P.copy_pad(b2, b);
            return b2;
        }
        View bt = P.talloc(cols_pad, rows_pad);
        P.transpose_into(bt, b);
        return bt;
    };
    bool ok = true;
    if (m == 0 || n == 0) {
        ok = true;
    } else if (k == 0) {
        P.memset0(Cv);
    } else if (direct) {
        View a2 = Av, c2 = Cv;
        if (!a_ok) { a2 = P.talloc(m, k); P.copy_pad(a2, Av); }
        if (!c_ok) c2 = P.talloc(m, n);
        View b2 = stage_b(Bv, k, n);
        if (L == 0 || algo == SW_ALGO_NAIVE) ok = P.gemm(a2, b2, c2, TGT_STORE);
        else if (L <= 3) ok = P.fused(a2, b2, c2, L);
        else {  // FP64 deeper than three levels: Table 2 (BDPZ) or Alg. 2 (Strassen) steps on top
            P.fused_below = 3;
            ok = P.product(a2, b2, c2, L);
        }
        if (!c_ok) P.copy_pad(Cv, c2);
    } else if (L > 5) {
        return fail(h, SW_EUNSUPPORTED, "materialised schedules stop at depth 5 (7^5 leaf launches); raise the cutoff");
    } else {
        // materialised schedules: halve exactly; FP32 column splits must stay 16-byte aligned
        const long long gm = 1LL << L, gk = (eb == 4 && !bf) ? 4LL << L : 1LL << L, gn = gk;
        const bool exact = m % gm == 0 && k % gk == 0 && n % gn == 0;
        const bool inpl = sched == SW_SCHED_IN_PLACE;
        if (exact && a_ok && c_ok && (eb == 8 || bf || Planner::vec_ok(Bv))) {
            View bs = Bv;
            if (P.bt) {
                if (inpl) { P.transpose_square(Bv); bs.rows = n; bs.cols = k; }  // B <- B^T in place
                else bs = stage_b(Bv, k, n);
            }
            ok = P.product(Av, bs, Cv, L);
        } else if (odd == SW_PEEL && a_ok && c_ok && (eb == 8 || bf || Planner::vec_ok(Bv))) {
            long long me = m / gm * gm, ke = k / gk * gk, ne = n / gn * gn;
            if (inpl) me = ke = ne = std::min(me, std::min(ke, ne));
            auto sub = [&](View v, long long r0, long long c0, long long rows, long long cols) {
                return Planner::sub(v, r0, c0, rows, cols, eb);
            };
            // edge products first (SIMT: thin, and they read the even blocks IN_PLACE overwrites)
            if (me < m) ok &= P.simt(sub(Av, me, 0, m - me, k), Bv, sub(Cv, me, 0, m - me, n), TGT_STORE);
            if (ne < n) ok &= P.simt(sub(Av, 0, 0, me, k), sub(Bv, 0, ne, k, n - ne), sub(Cv, 0, ne, me, n - ne),
                                     TGT_STORE);
            if (me > 0 && ne > 0) {
                if (ke > 0) {
                    View be = sub(Bv, 0, 0, ke, ne), bs = be;
                    if (P.bt) {
                        if (inpl) { P.transpose_square(be); bs.rows = (int)ne; bs.cols = (int)ke; }
                        else bs = stage_b(be, (int)ke, (int)ne);
                    }
                    ok &= P.product(sub(Av, 0, 0, me, ke), bs, sub(Cv, 0, 0, me, ne), L);
                } else {
                    P.memset0(sub(Cv, 0, 0, me, ne));
                }
                if (ke < k)
                    ok &= P.simt(sub(Av, 0, ke, me, k - ke), sub(Bv, ke, 0, k - ke, ne), sub(Cv, 0, 0, me, ne),
                                 ke > 0 ? TGT_ADD : TGT_STORE);
            }
        } else {
            // pad into aligned copies whose sizes halve exactly L times (zero fill, Sec. 3.1)
            int mp = (int)round_up(m, gm), kp = (int)round_up(k, gk), np = (int)round_up(n, gn);
            if (inpl) mp = kp = np = (int)round_up(std::max(m, std::max(k, n)), std::max(gm, gk));
            View a2 = P.talloc(mp, kp);
            P.copy_pad(a2, Av);
            View b2 = stage_b(Bv, kp, np);
            View c2 = P.talloc(mp, np);
            ok = P.product(a2, b2, c2, L);
            View cv = c2;
            cv.rows = m;
            cv.cols = n;
            P.copy_pad(Cv, cv);
        }
    }
    if (!ok) return fail(h, SW_ECUDA, P.err.empty() ? "planning failed" : P.err);
    plan->ws_need = P.ws_peak;
    return SW_OK;
}

static sw_status run_ops(sw_handle h, Plan* plan, cudaStream_t s, size_t first, size_t last) {
    char* blob = static_cast<char*>(plan->d_blob);
    for (size_t oi = first; oi < last && oi < plan->ops.size(); ++oi) {
        Op& o = plan->ops[oi];
        cudaError_t e = cudaSuccess;
        sw_handle_s::ProfRec rec = {(int)o.kind, nullptr, nullptr};
        if (h->prof) {
            rec.e0 = prof_event(h);
            rec.e1 = prof_event(h);
            cudaEventRecord(rec.e0, s);
        }
        switch (o.kind) {
            case OP_GEMM_TF32:
            {
                const CUtensorMap* gm = o.ngmaps ? reinterpret_cast<const CUtensorMap*>(blob + o.gmaps_off) : nullptr;
                const Leaf* lv = reinterpret_cast<const Leaf*>(blob + o.leaves_off);
                const Target* tv = reinterpret_cast<const Target*>(blob + o.targets_off);
                const CUtensorMap* tm = o.ntmaps ? reinterpret_cast<const CUtensorMap*>(blob + o.tmaps_off) : nullptr;
                unsigned* fl = o.nflags ? reinterpret_cast<unsigned*>(blob + o.flags_off) : nullptr;
                const int* il = (o.has_item_leaf || o.has_layout) ? reinterpret_cast<const int*>(blob + o.item_leaf_off)
                                                                  : nullptr;
                const int* it = o.has_layout ? reinterpret_cast<const int*>(blob + o.item_tile_off) : nullptr;
                e = o.nmaj ? launch_gemm_tf32n(o.bn, o.maps, gm, lv, o.nleaves, tv, tm, fl, o.items, h->d_err, h->sms,
                                               s, o.pair, il, it, o.units)
                           : launch_gemm_tf32(o.bn, o.maps, gm, lv, o.nleaves, tv, tm, fl, o.items, h->d_err,
                                              h->sms, s, o.pair, il);
            }
                break;
            case OP_GEMM_SIMT:
                e = launch_gemm_simt(o.eb, reinterpret_cast<const MatRef*>(blob + o.refs_off),
                                     reinterpret_cast<const Leaf*>(blob + o.leaves_off), o.nleaves,
                                     reinterpret_cast<const Target*>(blob + o.targets_off), o.items, h->sms * 8, o.wtile, s);
                break;
            case OP_TRANSPOSE:
                e = launch_transpose_pad(o.rows, o.cols, static_cast<float*>(o.z), o.ldz,
                                         static_cast<const float*>(o.x), o.ldx, o.src_rows, o.src_cols, s);
                break;
            case OP_TRANSPOSE_SQ:
                e = launch_transpose_inplace(o.rows, static_cast<float*>(o.z), o.ldz, s);
                break;
            case OP_BATCH_COPY:
                e = launch_batched_copy(reinterpret_cast<const CopyJob*>(blob + o.jobs_off), o.njobs, o.tiles,
                                        o.transpose, s);
                break;
            case OP_SPLIT:
                e = launch_split_bf16(o.rows, o.cols, static_cast<const float*>(o.x), o.ldx, o.z,
                                      const_cast<void*>(o.y), o.ldz, s);
                break;
            case OP_SPLIT_TF32:
                e = launch_split_tf32(o.rows, o.cols, static_cast<const float*>(o.x), o.ldx, static_cast<float*>(o.z),
                                      static_cast<float*>(const_cast<void*>(o.y)), o.ldz, s);
                break;
            case OP_GEMM_TF32X3:
                e = launch_gemm_tf32x3(o.bn, o.maps, nullptr, reinterpret_cast<const Leaf*>(blob + o.leaves_off),
                                       o.nleaves, reinterpret_cast<const Target*>(blob + o.targets_off),
                                       o.ntmaps ? reinterpret_cast<const CUtensorMap*>(blob + o.tmaps_off) : nullptr,
                                       o.nflags ? reinterpret_cast<unsigned*>(blob + o.flags_off) : nullptr,
                                       o.items, h->d_err, h->sms, s,
                                       o.has_item_leaf ? reinterpret_cast<const int*>(blob + o.item_leaf_off)
                                                       : nullptr);
                break;
            case OP_GEMM_BF16X3:
                e = launch_gemm_bf16x3(o.bn, o.maps, nullptr, reinterpret_cast<const Leaf*>(blob + o.leaves_off),
                                       o.nleaves, reinterpret_cast<const Target*>(blob + o.targets_off),
                                       o.ntmaps ? reinterpret_cast<const CUtensorMap*>(blob + o.tmaps_off) : nullptr,
                                       o.nflags ? reinterpret_cast<unsigned*>(blob + o.flags_off) : nullptr,
                                       o.items, h->d_err, h->sms, s,
                                       (o.has_item_leaf || o.has_layout)
                                           ? reinterpret_cast<const int*>(blob + o.item_leaf_off)
                                           : nullptr,
                                       o.has_layout ? reinterpret_cast<const int*>(blob + o.item_tile_off) : nullptr,
                                       o.units, o.pair);
                break;
            case OP_ADDSUB:
                e = launch_addsub(o.eb, o.rows, o.cols, o.z, o.ldz, o.x, o.ldx, o.y, o.ldy, o.sy, s);
                break;
            case OP_COPY_PAD:
                e = launch_copy_pad(o.eb, o.rows, o.cols, o.z, o.ldz, o.x, o.ldx, o.src_rows, o.src_cols, s);
                break;
            case OP_PREADD:
                e = o.pre_two ? launch_preadd2(o.pre, o.pre_b, s) : launch_preadd(o.eb, o.pre, s);
                break;
            case OP_PREADD_SPLIT:
                e = launch_preadd_split(o.pre, o.sout, o.pre_b, o.sout_b, s);
                break;
            case OP_MEMSET:
                e = cudaMemset2DAsync(o.z, (size_t)o.ldz * o.eb, 0, (size_t)o.cols * o.eb, (size_t)o.rows, s);
                break;
        }
        if (h->prof) {
            cudaEventRecord(rec.e1, s);
            h->prof_live.push_back(rec);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    }
    return SW_OK;
}

static sw_status run_plan(sw_handle h, Plan* plan, cudaStream_t s) {
    return run_ops(h, plan, s, 0, plan->ops.size());
}

// Run a plan: eagerly, or (batched plans, profiling off) through its captured CUDA graph.
static sw_status execute(sw_handle h, Plan* plan, cudaStream_t s) {
    if (!plan->use_graph || h->prof) return run_plan(h, plan, s);
    if (!plan->gexec) {
        if (!h->capture_stream &&
            cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "capture stream");
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
        sw_status st = run_plan(h, plan, h->capture_stream);
        e = cudaStreamEndCapture(h->capture_stream, &g);
        if (st != SW_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
        e = cudaGraphInstantiate(&plan->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { plan->gexec = nullptr; return cuda_fail(h, e, "graph instantiate"); }
    }
    cudaError_t e = cudaGraphLaunch(plan->gexec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    return SW_OK;
}

static sw_status build_batched_plan(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant,
                                    bool dry, Plan* plan, int bn = 256, bool pair = false) {
    Planner P;
    P.batch_bn = bn;
    P.batch_pair = pair;
    P.eb = 4;
    P.bf = false;
    P.nmaj = !tf32_bt_form();
    P.bt = !P.nmaj;
    P.variant = variant;
    P.dry = dry;
    P.ws_base = h->ws;
    P.plan = plan;
    P.sched = SW_SCHED_FUSED;
    P.algo = (int)(variant & SW_ALGO_MASK);
    std::vector<int> depth(count);
    int dmax = 0;
    for (int i = 0; i < count; ++i) {
        depth[i] = resolve_depth(probs[i].m, probs[i].n, probs[i].k, cutoff, variant, 4);
        dmax = std::max(dmax, depth[i]);
    }
    plan->depth = dmax;
    if (!P.batched(probs, count, depth)) return fail(h, SW_ECUDA, P.err.empty() ? "batched planning failed" : P.err);
    plan->ws_need = P.ws_peak;
    plan->use_graph = true;
    return SW_OK;
}

// Plan construction: a dry run sizes the workspace, the real run fills the plan, whose descriptors
// are uploaded once.  Growing the workspace flushes cached plans, so callers size every plan they
// will hold before building any of them.
using PlanBuilder = std::function<sw_status(bool dry, Plan* plan)>;

static sw_status plan_need(const PlanBuilder& build, size_t* need) {
    Plan d;
    sw_status st = build(true, &d);
    if (st == SW_OK) *need = d.ws_need;
    return st;
}

static sw_status plan_make(sw_handle h, const PlanBuilder& build, Plan** out) {
    Plan* plan = new Plan();
    sw_status st = build(false, plan);
    if (st != SW_OK) { delete plan; return st; }
    if (!plan->blob.empty()) {
        if (cudaMalloc(&plan->d_blob, plan->blob.size()) != cudaSuccess) {
            cudaGetLastError();
            delete plan;
            return fail(h, SW_ENOMEM, "descriptor allocation failed");
        }
        cudaMemcpy(plan->d_blob, plan->blob.data(), plan->blob.size(), cudaMemcpyHostToDevice);
    }
    *out = plan;
    return SW_OK;
}

static void plan_cache(sw_handle h, const std::string& key, Plan* plan) {
    if (h->plans.size() >= 256) flush_plans(h);
    h->plans[key] = plan;
}

static sw_status cached_plan(sw_handle h, const std::string& key, const PlanBuilder& build, Plan** out) {
    auto it = h->plans.find(key);
    if (it != h->plans.end()) { *out = it->second; return SW_OK; }
    size_t need = 0;
    sw_status st = plan_need(build, &need);
    if (st != SW_OK) return st;
    st = ensure_ws(h, need);
    if (st != SW_OK) return st;
    st = plan_make(h, build, out);
    if (st != SW_OK) return st;
    plan_cache(h, key, *out);
    return SW_OK;
}

// Device time of one run of a plan on `s` (after one untimed run), with the error word checked.
static sw_status time_plan(sw_handle h, Plan* plan, cudaStream_t s, double* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(h, cudaGetLastError(), "tuning events");
    }
    sw_status st = run_plan(h, plan, s);
    if (st == SW_OK) {
        cudaEventRecord(e0, s);
        st = run_plan(h, plan, s);
        cudaEventRecord(e1, s);
    }
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (st == SW_OK && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SW_OK) return st;
    if (e != cudaSuccess) return cuda_fail(h, e, "tuning run");
    int code = 0;
    e = cudaMemcpy(&code, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (code != 0) {
        cudaMemset(h->d_err, 0, sizeof(int));
        flush_plans(h);
        return fail(h, SW_ETIMEOUT, "bounded device wait expired while tuning (code " + std::to_string(code) + ")");
    }
    *ms = t;
    return SW_OK;
}

// Autotuner: time every candidate (each a builder for one configuration) on the caller's operands,
// keep the fastest plan under `key`, forget the others.  Returns the winner's index.
static sw_status tune(sw_handle h, const std::string& key, const std::vector<PlanBuilder>& cands, cudaStream_t s,
                      int* best, double* best_ms) {
    size_t need = 0;
    std::vector<char> ok(cands.size(), 0);
    for (size_t i = 0; i < cands.size(); ++i) {
        size_t b = 0;
        if (plan_need(cands[i], &b) == SW_OK) { ok[i] = 1; need = std::max(need, b); }
    }
    sw_status st = ensure_ws(h, need);  // sized for every candidate: no flush while tuning
    if (st != SW_OK) return st;
    Plan* keep = nullptr;
    *best = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (!ok[i]) continue;
        Plan* p = nullptr;
        if (plan_make(h, cands[i], &p) != SW_OK) continue;
        double t = 0.0;
        st = time_plan(h, p, s, &t);
        if (st != SW_OK) { delete p; delete keep; return st; }
        if (*best < 0 || t < *best_ms) {
            delete keep;
            keep = p;
            *best = (int)i;
            *best_ms = t;
        } else {
            delete p;
        }
    }
    if (!keep) return fail(h, SW_EUNSUPPORTED, "no tuning candidate could be planned");
    plan_cache(h, key, keep);
    return SW_OK;
}

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

static sw_status do_mm(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int m,
                       int n, int k, int cutoff, uint32_t variant, void* stream) {
    if (!h) return SW_EINVAL;
    if (m < 0 || n < 0 || k < 0) return fail(h, SW_EINVAL, "negative dimension");
    if ((m && k && !A) || (k && n && !B) || (m && n && !C)) return fail(h, SW_EINVAL, "null matrix pointer");
    if ((m && k && lda < std::max(k, 1)) || (k && n && ldb < std::max(n, 1)) || (m && n && ldc < std::max(n, 1)))
        return fail(h, SW_EINVAL, "leading dimension smaller than the row length");
    std::lock_guard<std::mutex> lock(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto builder = [=](int c) {
        return PlanBuilder([=](bool dry, Plan* p) {
            return build_plan(h, eb, A, lda, B, ldb, C, ldc, m, n, k, c, variant, dry, p);
        });
    };
    auto key_of = [&](int c) {
        char key[256];
        snprintf(key, sizeof(key), "%d|%p|%d|%p|%d|%p|%d|%d|%d|%d|%d|%u", eb, A, lda, B, ldb, C, ldc, m, n, k, c,
                 variant);
        return std::string(key);
    };
    // cutoff <= 0: the autotuner picks the depth on the first call for this shape and variant (not
    // under stream capture, and not for IN_PLACE, whose runs overwrite A and B)
    const uint32_t algo = variant & SW_ALGO_MASK, sched = variant & SW_SCHED_MASK;
    if (cutoff <= 0 && algo != SW_ALGO_NAIVE && sched != SW_SCHED_IN_PLACE && !capturing(s) && m && n && k) {
        char sig[160];
        const int align = (int)((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
                                 reinterpret_cast<uintptr_t>(C)) & 15) | (((lda | ldb | ldc) & 3) << 4);
        snprintf(sig, sizeof(sig), "M|%d|%d|%d|%d|%u|%d", eb, m, n, k, variant, align);
        auto t = h->tuned.find(sig);
        if (t != h->tuned.end()) {
            cutoff = t->second.cutoff;
        } else {
            // depths whose leaves stay large enough to keep the leaf kernels efficient
            const bool tc = eb == 4;
            const int leaf_min = tc ? 1024 : 128, lmax = sched == SW_SCHED_FUSED ? (tc ? 2 : 6) : 2;
            const int dmin = std::min(m, std::min(n, k));
            std::vector<int> cuts;
            for (int L = 0, prev = -1; L <= lmax && (dmin >> L) >= leaf_min; ++L) {
                const int c = (int)ceil_div(dmin, 1LL << L);
                const int d = resolve_depth(m, n, k, c, variant, eb);
                if (d != prev) cuts.push_back(c);
                prev = d;
            }
            // FP64: every level saves FP64 multiply-adds at little cost, so only the three deepest
            // depths are timed
            if (!tc && cuts.size() > 3) cuts.erase(cuts.begin(), cuts.end() - 3);
            if (cuts.size() >= 2) {
                std::vector<PlanBuilder> cands;
                for (int c : cuts) cands.push_back(builder(c));
                int best = -1;
                double ms = 0.0;
                sw_status st = tune(h, key_of(cuts[0]) + "|tuning", cands, s, &best, &ms);
                if (st != SW_OK) return st;
                // the winner's plan goes under its own key; it runs once more below, so C holds
                // exactly its result
                Plan* p = h->plans[key_of(cuts[0]) + "|tuning"];
                h->plans.erase(key_of(cuts[0]) + "|tuning");
                cutoff = cuts[best];
                plan_cache(h, key_of(cutoff), p);
                sw_handle_s::Tune tr;
                tr.cutoff = cutoff;
                tr.candidates = (int)cuts.size();
                tr.ms = ms;
                h->tuned[sig] = tr;
                h->last_tune = tr;
                h->has_tune = true;
            }
        }
    }
    Plan* plan = nullptr;
    sw_status st = cached_plan(h, key_of(cutoff), builder(cutoff), &plan);
    if (st != SW_OK) return st;
    return execute(h, plan, s);
}

// ====================================================================== serving loop
// A host thread admits submitted requests in arrival order while their workspace fits the arena
// and a completion slot is free.  Each admitted request is planned inside the arena.  When the
// plan ends in a grouped TF32 GEMM (BN 256, no ordering counters), every op before it runs on a
// side stream, and the GEMM's leaves, targets and tensor maps are appended to the descriptor
// arrays of the resident kernel, which claims the published tiles one by one on its share of the
// SMs; the request is complete when its counter reaches 4 per tile (one per epilogue warp).
// Other plans (FP64, split-BF16 leaves, padded or peeled shapes) run whole on a side stream with
// the SMs the resident kernel leaves free.
namespace {

constexpr int SRV_SIDE = 4;                   // side streams
constexpr unsigned SRV_MAX_ITEMS = 1u << 21;  // published tiles per generation
constexpr int SRV_MAX_LEAVES = 1 << 16;
constexpr int SRV_MAX_TARGETS = 1 << 18;
constexpr int SRV_MAX_MAPS = 1 << 14;   // operand tensor maps
constexpr int SRV_MAX_TMAPS = 1 << 16;  // target tensor maps
constexpr size_t SRV_BLOB_BYTES = 256u << 20;
constexpr size_t SRV_ALIGN = 1024;

enum ReqState { RQ_QUEUED = 0, RQ_PRE = 1, RQ_PUBLISHED = 2, RQ_DONE = 3 };

struct ServerReq {
    uint64_t ticket = 0;
    sw_request req;
    size_t need = 0;      // arena bytes of the workspace
    size_t ws_off = 0, blob_off = 0, blob_bytes = 0;
    Plan plan;
    int slot = -1;
    bool resident = false;
    unsigned items = 0;   // resident tiles
    int state = RQ_QUEUED;
    cudaEvent_t ev = nullptr;
    sw_status status = SW_OK;
    std::string msg;
};

// The resident kernel's descriptors for one appended GEMM (indices already rebased).
struct AppendSet {
    std::vector<Leaf> leaves;
    std::vector<Target> targets;
    std::vector<CUtensorMap> maps, tmaps;
    std::vector<int> item_leaf;
};

}  // namespace

struct Server {
    sw_handle_s shadow;  // planning errors and side-stream launches (grid: the SMs left free)
    sw_server_cfg cfg{};
    int device = 0, sms = 0;
    std::thread thr;
    // guarded by mu: the queue, the ticket map, every request's state / status, quit, dead
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool quit = false;
    sw_status dead = SW_OK;
    std::string dead_msg;
    std::deque<ServerReq*> queue;
    std::unordered_map<uint64_t, ServerReq*> reqs;
    uint64_t next_ticket = 1;
    // server-thread state
    std::vector<ServerReq*> active;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> ev_pool;
    Arena arena, blobs;
    int side_rr = 0;
    unsigned n_items = 0;
    int n_leaves = 0, n_targets = 0, n_maps = 0, n_tmaps = 0;
    bool res_launched = false;
    // device memory
    char* arena_mem = nullptr;
    char* blob_mem = nullptr;
    char* desc_mem = nullptr;
    CUtensorMap* gmaps_d = nullptr;
    CUtensorMap* tmaps_d = nullptr;
    Leaf* leaves_d = nullptr;
    Target* targets_d = nullptr;
    int* item_leaf_d = nullptr;
    unsigned* ctl_d = nullptr;     // [0] next unclaimed tile, [16] error word, [32 ...] done counters
    unsigned* poll_h = nullptr;    // pinned host copy of ctl_d
    unsigned* mapped_h = nullptr;  // host-mapped: [0] published tiles, [32] stop
    unsigned* mapped_d = nullptr;
    cudaStream_t res_stream = nullptr, ctl_stream = nullptr, side[SRV_SIDE] = {};
    cudaEvent_t res_ev = nullptr;

    size_t ctl_bytes() const { return 128 + 4 * (size_t)cfg.max_inflight; }
    int* err_d() const { return reinterpret_cast<int*>(ctl_d + 16); }
    unsigned* done_d() const { return ctl_d + 32; }
    void set_mapped(int i, unsigned v) {
        std::atomic_thread_fence(std::memory_order_seq_cst);
        reinterpret_cast<volatile unsigned*>(mapped_h)[i] = v;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }

    sw_status init(sw_handle h, const sw_server_cfg* c, std::string* msg);
    void release_device();
    void loop();
    void start(ServerReq* r);
    bool step();
    bool append(ServerReq* r, bool* fits);
    void publish() { cudaStreamSynchronize(ctl_stream); set_mapped(0, n_items); }
    bool kernel_running() { return res_launched && cudaEventQuery(res_ev) == cudaErrorNotReady; }
    sw_status launch_resident();
    void stop_kernel();
    void reset_generation();
    void complete(ServerReq* r, sw_status st, const std::string& msg);
    void fail_all(sw_status st, const std::string& msg);
    void fatal(const std::string& msg);
    cudaEvent_t take_event() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }
};

// The resident kernel runs the BN = 256 TF32 grouped GEMM only, with operand maps passed by value
// in the op (re-homed to global memory) and no ordering counters.
static bool resident_form(const Plan& p) {
    if (p.ops.empty()) return false;
    const Op& o = p.ops.back();
    return o.kind == OP_GEMM_TF32 && o.nmaj == !tf32_bt_form() && !o.pair && o.bn == 256 && o.nflags == 0 &&
           o.ngmaps == 0 && o.items > 0 &&
           o.nleaves > 0 && (unsigned)o.items <= SRV_MAX_ITEMS / 2 && o.nleaves <= SRV_MAX_LEAVES / 2 &&
           o.ntmaps <= SRV_MAX_TMAPS / 2;
}

sw_status Server::init(sw_handle h, const sw_server_cfg* c, std::string* msg) {
    device = h->device;
    sms = h->sms;
    if (c) cfg = *c;
    if (cfg.sm_share <= 0) cfg.sm_share = std::max(1, sms - 16);
    cfg.sm_share = std::min(cfg.sm_share, std::max(1, sms - 4));
    if (cfg.max_inflight <= 0) cfg.max_inflight = 64;
    cfg.max_inflight = std::min(cfg.max_inflight, 4096);
    if (cfg.idle_us <= 0) cfg.idle_us = 20000;
    cfg.idle_us = std::min(cfg.idle_us, 1000000);  // well inside the kernel's 2 s bounded waits
    if (cfg.budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        cfg.budget_bytes = std::min((size_t)60 << 30, fr / 4 * 3);
    }
    cfg.budget_bytes = (size_t)round_up((long long)cfg.budget_bytes, (long long)SRV_ALIGN);
    shadow.device = device;
    shadow.sms = std::max(1, sms - cfg.sm_share);
    auto oom = [&](const char* what) {
        cudaGetLastError();
        *msg = std::string("serving: allocation of ") + what + " failed";
        release_device();
        return SW_ENOMEM;
    };
    if (cudaMalloc(&arena_mem, cfg.budget_bytes) != cudaSuccess) return oom("the workspace arena");
    arena.init(cfg.budget_bytes);
    if (cudaMalloc(&blob_mem, SRV_BLOB_BYTES) != cudaSuccess) return oom("the descriptor pool");
    blobs.init(SRV_BLOB_BYTES);
    const size_t desc_bytes = (size_t)SRV_MAX_MAPS * 128 + (size_t)SRV_MAX_TMAPS * 128 +
                              (size_t)SRV_MAX_LEAVES * sizeof(Leaf) + (size_t)SRV_MAX_TARGETS * sizeof(Target) +
                              (size_t)SRV_MAX_ITEMS * 4 + 4 * SRV_ALIGN;
    if (cudaMalloc(&desc_mem, desc_bytes) != cudaSuccess) return oom("the resident descriptors");
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        char* p = desc_mem + off;
        off = (size_t)round_up((long long)(off + bytes), (long long)SRV_ALIGN);
        return p;
    };
    gmaps_d = reinterpret_cast<CUtensorMap*>(carve((size_t)SRV_MAX_MAPS * 128));
    tmaps_d = reinterpret_cast<CUtensorMap*>(carve((size_t)SRV_MAX_TMAPS * 128));
    leaves_d = reinterpret_cast<Leaf*>(carve((size_t)SRV_MAX_LEAVES * sizeof(Leaf)));
    targets_d = reinterpret_cast<Target*>(carve((size_t)SRV_MAX_TARGETS * sizeof(Target)));
    item_leaf_d = reinterpret_cast<int*>(carve((size_t)SRV_MAX_ITEMS * 4));
    if (cudaMalloc(&ctl_d, ctl_bytes()) != cudaSuccess) return oom("the control words");
    if (cudaMemset(ctl_d, 0, ctl_bytes()) != cudaSuccess) return oom("the control words");
    shadow.d_err = err_d();
    if (cudaHostAlloc(&poll_h, ctl_bytes(), cudaHostAllocDefault) != cudaSuccess) return oom("the poll buffer");
    if (cudaHostAlloc(&mapped_h, 256, cudaHostAllocMapped) != cudaSuccess) return oom("the mapped words");
    memset(mapped_h, 0, 256);
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&mapped_d), mapped_h, 0) != cudaSuccess)
        return oom("the mapped words (device view)");
    if (cudaStreamCreateWithFlags(&res_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctl_stream, cudaStreamNonBlocking) != cudaSuccess)
        return oom("streams");
    for (auto& s : side)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return oom("streams");
    if (cudaEventCreateWithFlags(&res_ev, cudaEventDisableTiming) != cudaSuccess) return oom("events");
    for (int i = cfg.max_inflight - 1; i >= 0; --i) free_slots.push_back(i);
    return SW_OK;
}

void Server::release_device() {
    cudaGetLastError();
    if (res_stream) cudaStreamSynchronize(res_stream);
    for (auto s : side)
        if (s) cudaStreamSynchronize(s);
    if (ctl_stream) cudaStreamSynchronize(ctl_stream);
    for (auto e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    if (res_ev) cudaEventDestroy(res_ev);
    for (auto& s : side)
        if (s) { cudaStreamDestroy(s); s = nullptr; }
    if (res_stream) cudaStreamDestroy(res_stream);
    if (ctl_stream) cudaStreamDestroy(ctl_stream);
    if (mapped_h) cudaFreeHost(mapped_h);
    if (poll_h) cudaFreeHost(poll_h);
    if (ctl_d) cudaFree(ctl_d);
    if (desc_mem) cudaFree(desc_mem);
    if (blob_mem) cudaFree(blob_mem);
    if (arena_mem) cudaFree(arena_mem);
    res_ev = nullptr;
    res_stream = ctl_stream = nullptr;
    mapped_h = poll_h = ctl_d = nullptr;
    desc_mem = blob_mem = arena_mem = nullptr;
}

void Server::complete(ServerReq* r, sw_status st, const std::string& msg) {
    arena.release(r->ws_off, r->need);
    if (r->blob_bytes) blobs.release(r->blob_off, r->blob_bytes);
    r->blob_bytes = 0;
    if (r->slot >= 0) free_slots.push_back(r->slot);
    r->slot = -1;
    if (r->ev) { ev_pool.push_back(r->ev); r->ev = nullptr; }
    active.erase(std::remove(active.begin(), active.end(), r), active.end());
    std::lock_guard<std::mutex> lk(mu);
    r->status = st;
    r->msg = msg;
    r->state = RQ_DONE;  // a waiter may free r from here on
    cv_done.notify_all();
}

// Fail every admitted request once no work of theirs can still be in flight.
void Server::fail_all(sw_status st, const std::string& msg) {
    if (res_launched) {
        set_mapped(32, 1u);
        cudaEventSynchronize(res_ev);
        set_mapped(32, 0u);
    }
    for (auto s : side) cudaStreamSynchronize(s);
    std::vector<ServerReq*> all = active;
    for (ServerReq* r : all) complete(r, st, msg);
}

void Server::fatal(const std::string& msg) {
    fail_all(SW_ECUDA, msg);
    std::lock_guard<std::mutex> lk(mu);
    dead = SW_ECUDA;
    dead_msg = msg;
}

// Ask the resident kernel to exit once every published tile is claimed, and wait for it.
void Server::stop_kernel() {
    if (!res_launched) return;
    set_mapped(32, 1u);
    cudaEventSynchronize(res_ev);  // its waits are bounded, so this ends
    set_mapped(32, 0u);
}

// Start a new generation of descriptor arrays: only while no resident kernel runs.
void Server::reset_generation() {
    cudaMemsetAsync(ctl_d, 0, 4, ctl_stream);
    cudaStreamSynchronize(ctl_stream);
    set_mapped(0, 0u);
    n_items = 0;
    n_leaves = n_targets = n_maps = n_tmaps = 0;
}

sw_status Server::launch_resident() {
    set_mapped(32, 0u);
    ResidentCtl c;
    c.next = ctl_d;
    c.published = mapped_d;
    c.stop = mapped_d + 32;
    c.item_leaf = item_leaf_d;
    c.done = done_d();
    c.idle_ns = (unsigned long long)cfg.idle_us * 1000ull;
    cudaError_t e = launch_gemm_tf32_resident(gmaps_d, leaves_d, targets_d, tmaps_d, c, err_d(), cfg.sm_share,
                                              res_stream, !tf32_bt_form());
    if (e != cudaSuccess) return SW_ECUDA;
    cudaEventRecord(res_ev, res_stream);
    res_launched = true;
    return SW_OK;
}

void Server::start(ServerReq* r) {
    active.push_back(r);
    const sw_request& q = r->req;
    shadow.last_error.clear();
    sw_status st = build_plan(&shadow, q.elem_bytes, q.A, q.lda, q.B, q.ldb, q.C, q.ldc, q.m, q.n, q.k, q.cutoff,
                              q.variant, false, &r->plan, arena_mem + r->ws_off, true);
    r->plan.owns_blob = false;
    if (st != SW_OK) { complete(r, st, shadow.last_error); return; }
    if (r->plan.ws_need > r->need) { complete(r, SW_ECUDA, "serving: workspace grew after sizing"); return; }
    cudaStream_t s = side[side_rr];
    side_rr = (side_rr + 1) % SRV_SIDE;
    if (!r->plan.blob.empty()) {
        const size_t nb = (size_t)round_up((long long)r->plan.blob.size(), 256);
        size_t off = 0;
        if (!blobs.alloc(nb, &off)) { complete(r, SW_EBUDGET, "serving: descriptor pool full"); return; }
        r->blob_off = off;
        r->blob_bytes = nb;
        r->plan.d_blob = blob_mem + off;
        cudaMemcpyAsync(r->plan.d_blob, r->plan.blob.data(), r->plan.blob.size(), cudaMemcpyHostToDevice, s);
    }
    r->resident = resident_form(r->plan);
    st = run_ops(&shadow, &r->plan, s, 0, r->plan.ops.size() - (r->resident ? 1 : 0));
    if (st != SW_OK) {
        cudaStreamSynchronize(s);
        complete(r, st, shadow.last_error);
        return;
    }
    r->ev = take_event();
    cudaEventRecord(r->ev, s);
    std::lock_guard<std::mutex> lk(mu);
    r->state = RQ_PRE;
}

// Append the request's final GEMM to the resident descriptor arrays (fresh 128-byte lines, so
// no line the kernel may hold cached changes).  *fits = false: no room in this generation.
bool Server::append(ServerReq* r, bool* fits) {
    const Op& o = r->plan.ops.back();
    const uint8_t* blob = r->plan.blob.data();
    const Leaf* lv = reinterpret_cast<const Leaf*>(blob + o.leaves_off);
    const Target* tv = reinterpret_cast<const Target*>(blob + o.targets_off);
    const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(blob + o.tmaps_off);
    int ntg = 0, nmp = 0;
    for (int i = 0; i < o.nleaves; ++i) {
        ntg = std::max(ntg, lv[i].tgt_begin + lv[i].tgt_count);
        nmp = std::max(nmp, std::max(lv[i].a_map, lv[i].b_map) + 1);
    }
    const int L0 = (int)round_up(n_leaves, 2), T0 = (int)round_up(n_targets, 8), M0 = n_maps, TM0 = n_tmaps;
    const unsigned I0 = n_items;
    *fits = L0 + o.nleaves <= SRV_MAX_LEAVES && T0 + ntg <= SRV_MAX_TARGETS && M0 + nmp <= SRV_MAX_MAPS &&
            TM0 + o.ntmaps <= SRV_MAX_TMAPS && (unsigned long long)I0 + o.items <= SRV_MAX_ITEMS;
    if (!*fits) return false;
    AppendSet a;
    a.maps.assign(o.maps.m, o.maps.m + nmp);
    a.tmaps.assign(tm, tm + o.ntmaps);
    a.targets.assign(tv, tv + ntg);
    for (Target& t : a.targets)
        if (t.map >= 0) t.map += TM0;
    a.item_leaf.assign(o.items, -1);
    for (int i = 0; i < o.nleaves; ++i) {
        Leaf lf = lv[i];
        const long long tiles = ceil_div(lf.m, tf32_tile_m()) * lf.tiles_n;
        for (long long t = 0; t < tiles; ++t) {
            const long long it = lf.tile_begin + t;
            if (it < 0 || it >= o.items) return false;
            a.item_leaf[it] = L0 + i;
        }
        lf.a_map += M0;
        lf.b_map += M0;
        lf.tgt_begin += T0;
        lf.tile_begin += (int)I0;
        lf.tag = r->slot;
        a.leaves.push_back(lf);
    }
    for (int v : a.item_leaf)
        if (v < 0) return false;
    cudaStream_t s = ctl_stream;
    cudaMemcpyAsync(gmaps_d + M0, a.maps.data(), a.maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s);
    if (!a.tmaps.empty())
        cudaMemcpyAsync(tmaps_d + TM0, a.tmaps.data(), a.tmaps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                        s);
    cudaMemcpyAsync(leaves_d + L0, a.leaves.data(), a.leaves.size() * sizeof(Leaf), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(targets_d + T0, a.targets.data(), a.targets.size() * sizeof(Target), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(item_leaf_d + I0, a.item_leaf.data(), a.item_leaf.size() * sizeof(int), cudaMemcpyHostToDevice,
                    s);
    cudaMemsetAsync(done_d() + r->slot, 0, 4, s);
    cudaStreamSynchronize(s);  // the staging vectors die with this frame
    n_leaves = L0 + o.nleaves;
    n_targets = T0 + ntg;
    n_maps = M0 + nmp;
    n_tmaps = TM0 + o.ntmaps;
    n_items = I0 + (unsigned)o.items;
    r->items = (unsigned)o.items;
    return true;
}

// One pass of the loop over admitted requests; returns whether anything moved.
bool Server::step() {
    std::vector<ServerReq*> ready, published;
    for (ServerReq* r : active) {
        if (r->state == RQ_PRE) {
            const cudaError_t e = cudaEventQuery(r->ev);
            if (e == cudaSuccess) ready.push_back(r);
            else if (e != cudaErrorNotReady) { fatal(std::string("serving: ") + cudaGetErrorString(e)); return true; }
        } else if (r->state == RQ_PUBLISHED) {
            published.push_back(r);
        }
    }
    if (ready.empty() && published.empty()) return false;
    // kernel state first, then the counters: after an exit the counters are final
    bool exited = false;
    if (res_launched) {
        const cudaError_t e = cudaEventQuery(res_ev);
        if (e == cudaSuccess) exited = true;
        else if (e != cudaErrorNotReady) { fatal(std::string("serving: ") + cudaGetErrorString(e)); return true; }
    }
    const unsigned pub_at_poll = n_items;
    cudaMemcpyAsync(poll_h, ctl_d, ctl_bytes(), cudaMemcpyDeviceToHost, ctl_stream);
    const cudaError_t pe = cudaStreamSynchronize(ctl_stream);
    if (pe != cudaSuccess) { fatal(std::string("serving: ") + cudaGetErrorString(pe)); return true; }
    const int errw = (int)poll_h[16];
    if (errw != 0) {
        fail_all(errw == ERR_ALIGN ? SW_ECUDA : SW_ETIMEOUT,
                 "serving: device error code " + std::to_string(errw) + " (a bounded wait expired or a TMA "
                 "coordinate was misaligned); every request in flight was failed");
        cudaMemsetAsync(err_d(), 0, 4, ctl_stream);
        reset_generation();
        return true;
    }
    bool moved = false;
    const unsigned next = poll_h[0];
    for (ServerReq* r : published) {
        if (poll_h[32 + r->slot] >= 4u * r->items) {
            complete(r, SW_OK, "");
            moved = true;
        } else if (exited && next >= pub_at_poll) {
            complete(r, SW_ECUDA, "serving: the resident kernel exited with tiles of this request unreported");
            moved = true;
        }
    }
    bool appended = false, deferred = false;
    for (ServerReq* r : ready) {
        if (!r->resident) {
            complete(r, SW_OK, "");
            moved = true;
            continue;
        }
        bool fits = true;
        if (append(r, &fits)) {
            std::lock_guard<std::mutex> lk(mu);
            r->state = RQ_PUBLISHED;
            appended = moved = true;
        } else if (fits) {
            complete(r, SW_ECUDA, "serving: inconsistent leaf descriptors");
            moved = true;
        } else {
            deferred = true;
        }
    }
    if (appended) publish();
    bool pending = false;
    for (ServerReq* r : active) pending |= r->state == RQ_PUBLISHED;
    if (pending) {
        if (!kernel_running()) {
            if (launch_resident() != SW_OK) { fatal("serving: resident kernel launch failed"); return true; }
            moved = true;
        }
    } else if (n_items > 0 && (deferred || !kernel_running())) {
        stop_kernel();
        reset_generation();
        moved = true;
    }
    return moved;
}

void Server::loop() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<ServerReq*> incoming;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty() && queue.empty()) {
                if (quit) break;
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
            // admission in arrival order: stop at the first request that does not fit
            while (!queue.empty() && !free_slots.empty()) {
                ServerReq* r = queue.front();
                if (dead == SW_OK) {
                    size_t off = 0;
                    if (!arena.alloc(r->need, &off)) break;
                    r->ws_off = off;
                    r->slot = free_slots.back();
                    free_slots.pop_back();
                } else {
                    r->need = 0;
                }
                queue.pop_front();
                incoming.push_back(r);
            }
        }
        for (ServerReq* r : incoming) {
            if (dead == SW_OK) start(r);
            else { active.push_back(r); complete(r, dead, dead_msg); }
        }
        if (!step() && incoming.empty()) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    stop_kernel();
}

// ====================================================================== C ABI
extern "C" {

sw_status sw_create(sw_handle* out, size_t budget) {
    if (!out) return SW_EINVAL;
    *out = nullptr;
    sw_handle h = new sw_handle_s();
    h->budget = budget;
    if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); delete h; return SW_ECUDA; }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (cudaMalloc(&h->d_err, 256) != cudaSuccess) { cudaGetLastError(); delete h; return SW_ENOMEM; }
    cudaMemset(h->d_err, 0, 256);
    h->d_norms = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->d_err) + 64);
    if (!encode_fn()) { cudaFree(h->d_err); delete h; return SW_ECUDA; }
    *out = h;
    return SW_OK;
}

sw_status sw_destroy(sw_handle h) {
    if (!h) return SW_EINVAL;
    cudaSetDevice(h->device);
    if (h->server) sw_server_stop(h);
    cudaDeviceSynchronize();
    for (auto& kv : h->plans) delete kv.second;
    h->plans.clear();
    if (h->ws) cudaFree(h->ws);
    if (h->io) cudaFree(h->io);
    if (h->d_err) cudaFree(h->d_err);
    for (auto& r : h->prof_live) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto e : h->prof_free) cudaEventDestroy(e);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->io_in) cudaStreamDestroy(h->io_in);
    if (h->io_out) cudaStreamDestroy(h->io_out);
    for (auto e : h->io_ev) cudaEventDestroy(e);
    delete h;
    return SW_OK;
}

const char* sw_last_error(sw_handle h) { return h ? h->last_error.c_str() : "null handle"; }

sw_status sw_mm_depth(int m, int n, int k, int cutoff, uint32_t variant, int elem_bytes, int* depth) {
    if (!depth || m < 0 || n < 0 || k < 0 || (elem_bytes != 4 && elem_bytes != 8)) return SW_EINVAL;
    *depth = resolve_depth(m, n, k, cutoff, variant, elem_bytes);
    return SW_OK;
}

sw_status sw_mm_workspace_size(int m, int n, int k, int cutoff, uint32_t variant, int elem_bytes, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || k < 0 || (elem_bytes != 4 && elem_bytes != 8)) return SW_EINVAL;
    sw_handle_s tmp;
    Plan p;
    // sizes only: aligned dummy pointers and tight leading dimensions
    char* d = reinterpret_cast<char*>(static_cast<uintptr_t>(1) << 20);
    sw_status st = build_plan(&tmp, elem_bytes, d, std::max(k, 1), d, std::max(n, 1), d, std::max(n, 1), m, n, k,
                              cutoff, variant, true, &p);
    if (st != SW_OK) return st;
    *bytes = p.ws_need;
    return SW_OK;
}

sw_status sw_smm(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m, int n,
                 int k, int cutoff, uint32_t variant, void* stream) {
    return do_mm(h, 4, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream);
}

sw_status sw_dmm(sw_handle h, const double* A, int lda, const double* B, int ldb, double* C, int ldc, int m, int n,
                 int k, int cutoff, uint32_t variant, void* stream) {
    return do_mm(h, 8, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream);
}

sw_status sw_mm_batched(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant, void* stream) {
    if (!h) return SW_EINVAL;
    if (count < 0 || (count > 0 && !probs)) return fail(h, SW_EINVAL, "bad problem list");
    if ((variant & SW_SCHED_MASK) != SW_SCHED_FUSED || (variant & SW_LEAF_MASK) != SW_LEAF_TF32)
        return fail(h, SW_EUNSUPPORTED, "batched products take the FUSED schedule with TF32 leaves");
    if ((variant & SW_ALGO_MASK) > SW_ALGO_WINOGRAD_KNUTH) return fail(h, SW_EINVAL, "unknown algorithm bits");
    for (int i = 0; i < count; ++i) {
        const sw_problem& q = probs[i];
        if (q.m < 0 || q.n < 0 || q.k < 0) return fail(h, SW_EINVAL, "negative dimension in problem " + std::to_string(i));
        if ((q.m && q.k && (!q.A || q.lda < q.k)) || (q.k && q.n && (!q.B || q.ldb < q.n)) ||
            (q.m && q.n && (!q.C || q.ldc < q.n)))
            return fail(h, SW_EINVAL, "bad pointer or leading dimension in problem " + std::to_string(i));
    }
    if (count == 0) return SW_OK;
    std::lock_guard<std::mutex> lock(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // plan key: the problem list's bytes
    std::string key = "B|" + std::to_string(count) + "|" + std::to_string(cutoff) + "|" + std::to_string(variant) + "|";
    key.append(reinterpret_cast<const char*>(probs), sizeof(sw_problem) * (size_t)count);
    struct Cfg { int bn, pair, cutoff; };
    auto builder = [=](Cfg c) {
        return PlanBuilder([=](bool dry, Plan* p) {
            return build_batched_plan(h, count, probs, c.cutoff, variant, dry, p, c.bn, c.pair != 0);
        });
    };
    auto key_of = [&](Cfg c) {
        return key + "|" + std::to_string(c.bn) + "|" + std::to_string(c.pair) + "|" + std::to_string(c.cutoff);
    };
    Cfg cfg = {256, 0, cutoff};
    // cutoff <= 0: the autotuner times the grouped launch's tile shape (128- or 256-wide tiles on one
    // CTA, 256 x 256 tiles on CTA pairs) and the recursion cutoff on this problem list, once
    if (cutoff <= 0 && !capturing(s)) {
        auto t = h->tuned.find(key);
        if (t != h->tuned.end()) {
            cfg = {t->second.bn, t->second.pair, t->second.cutoff};
        } else {
            const int none = 1 << 30;  // no recursion
            std::vector<Cfg> cs = {{256, 0, none}, {128, 0, none}};
            if (!tf32_bt_form()) {     // CTA pairs need N-major B
                cs.push_back({256, 1, none});
                cs.push_back({256, 1, 2048});
            }
            std::vector<PlanBuilder> cands;
            for (const Cfg& c : cs) cands.push_back(builder(c));
            int best = -1;
            double ms = 0.0;
            sw_status st = tune(h, key + "|tuning", cands, s, &best, &ms);
            if (st != SW_OK) return st;
            cfg = cs[best];
            Plan* p = h->plans[key + "|tuning"];
            h->plans.erase(key + "|tuning");
            plan_cache(h, key_of(cfg), p);
            sw_handle_s::Tune tr;
            tr.cutoff = cfg.cutoff;
            tr.bn = cfg.bn;
            tr.pair = cfg.pair;
            tr.candidates = (int)cs.size();
            tr.ms = ms;
            h->tuned[key] = tr;
            h->last_tune = tr;
            h->has_tune = true;
        }
    }
    Plan* plan = nullptr;
    sw_status st = cached_plan(h, key_of(cfg), builder(cfg), &plan);
    if (st != SW_OK) return st;
    return execute(h, plan, s);
}

sw_status sw_last_tuning(sw_handle h, int* cutoff, int* tile_n, int* cta_pair, double* ms, int* candidates) {
    if (!h) return SW_EINVAL;
    std::lock_guard<std::mutex> lock(h->mu);
    if (!h->has_tune) return fail(h, SW_EINVAL, "nothing tuned on this handle yet");
    if (cutoff) *cutoff = h->last_tune.cutoff;
    if (tile_n) *tile_n = h->last_tune.bn;
    if (cta_pair) *cta_pair = h->last_tune.pair;
    if (ms) *ms = h->last_tune.ms;
    if (candidates) *candidates = h->last_tune.candidates;
    return SW_OK;
}

// Host-operand product in row panels of height mp (the last one lower): B goes over first, then
// panel i of A on the copy-in stream; panel i of C = A_i B runs on the caller's stream at the
// whole product's depth L (the panel's cutoff is its own smallest block side at depth L, which
// gives exactly L levels while that side is >= 2); panel i of C comes back on the copy-out stream
// while later panels still arrive and compute.  Row panels keep every copy one contiguous run.
static sw_status host_panels(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m,
                             int n, int k, int cutoff, uint32_t variant, int L, int mp, float* dA, long long lda2,
                             float* dB, long long ldb2, float* dC, long long ldc2, cudaStream_t s) {
    const int npan = (int)ceil_div(m, mp);
    {
        std::lock_guard<std::mutex> lock(h->mu);
        cudaSetDevice(h->device);
        if (!h->io_in && cudaStreamCreateWithFlags(&h->io_in, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "copy stream");
        if (!h->io_out && cudaStreamCreateWithFlags(&h->io_out, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "copy stream");
        while ((int)h->io_ev.size() < 2 * npan + 2) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                return cuda_fail(h, cudaGetLastError(), "copy event");
            h->io_ev.push_back(ev);
        }
    }
    cudaEvent_t* ev = h->io_ev.data();  // [0] start, [1 + i] A_i arrived, [1 + npan + i] C_i done, [last] out done
    // the call is synchronous: on any failure the copies already queued finish before it returns,
    // so the caller may release its host buffers
    auto drained = [&](sw_status st) {
        cudaStreamSynchronize(h->io_in);
        cudaStreamSynchronize(h->io_out);
        return st;
    };
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_in, ev[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dB, ldb2 * 4, B, (size_t)ldb * 4, (size_t)n * 4, k, cudaMemcpyHostToDevice, h->io_in);
    for (int i = 0; i < npan && e == cudaSuccess; ++i) {
        const int r0 = i * mp, hgt = std::min(mp, m - r0);
        e = cudaMemcpy2DAsync(dA + r0 * lda2, lda2 * 4, A + (size_t)r0 * lda, (size_t)lda * 4, (size_t)k * 4, hgt,
                              cudaMemcpyHostToDevice, h->io_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + i], h->io_in);
    }
    if (e != cudaSuccess) return drained(cuda_fail(h, e, "host to device copy"));
    for (int i = 0; i < npan; ++i) {
        const int r0 = i * mp, hgt = std::min(mp, m - r0);
        e = cudaStreamWaitEvent(s, ev[1 + i], 0);
        if (e != cudaSuccess) return drained(cuda_fail(h, e, "panel order"));
        int cut = cutoff;
        if ((variant & SW_ALGO_MASK) != SW_ALGO_NAIVE) {
            const long long d = 1LL << L;
            cut = (int)std::min(std::min(ceil_div(hgt, d), ceil_div(n, d)), ceil_div(k, d));
            if (cut < 2 || resolve_depth(hgt, n, k, cut, variant, 4) != L) cut = cutoff;  // low last panel
        }
        sw_status st = sw_smm(h, dA + r0 * lda2, (int)lda2, dB, (int)ldb2, dC + r0 * ldc2, (int)ldc2, hgt, n, k, cut,
                              variant, s);
        if (st != SW_OK) return drained(st);
        e = cudaEventRecord(ev[1 + npan + i], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_out, ev[1 + npan + i], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(C + (size_t)r0 * ldc, (size_t)ldc * 4, dC + r0 * ldc2, ldc2 * 4, (size_t)n * 4, hgt,
                                  cudaMemcpyDeviceToHost, h->io_out);
        if (e != cudaSuccess) return drained(cuda_fail(h, e, "device to host copy"));
    }
    e = cudaEventRecord(ev[1 + 2 * npan], h->io_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1 + 2 * npan], 0);
    if (e != cudaSuccess) return drained(cuda_fail(h, e, "panel order"));
    return sw_sync(h, s);
}

sw_status sw_smm_host(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m, int n,
                      int k, int cutoff, uint32_t variant, void* stream) {
    if (!h) return SW_EINVAL;
    if (m < 0 || n < 0 || k < 0 || (m && k && (!A || lda < k)) || (k && n && (!B || ldb < n)) ||
        (m && n && (!C || ldc < n)))
        return fail(h, SW_EINVAL, "bad host operand");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long lda2 = round_up(std::max(k, 1), 4), ldb2 = round_up(std::max(n, 1), 4), ldc2 = ldb2;
    const size_t ba = (size_t)round_up((long long)m * lda2 * 4, 256), bb = (size_t)round_up((long long)k * ldb2 * 4, 256),
                 bc = (size_t)round_up((long long)m * ldc2 * 4, 256);
    {
        std::lock_guard<std::mutex> lock(h->mu);
        cudaSetDevice(h->device);
        if (ba + bb + bc > h->io_bytes) {
            flush_plans(h);
            if (h->io) { cudaDeviceSynchronize(); cudaFree(h->io); h->io = nullptr; h->io_bytes = 0; }
            if (cudaMalloc(&h->io, ba + bb + bc) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, SW_ENOMEM, "host-path buffers");
            }
            h->io_bytes = ba + bb + bc;
        }
    }
    float* dA = reinterpret_cast<float*>(h->io);
    float* dB = reinterpret_cast<float*>(h->io + ba);
    float* dC = reinterpret_cast<float*>(h->io + ba + bb);
    cudaError_t e = cudaSuccess;
    // large FUSED / naive products with a given cutoff: A and C move in row panels so the copies
    // overlap the panel products and each other (the link is duplex)
    const uint32_t algo = variant & SW_ALGO_MASK, sched = variant & SW_SCHED_MASK;
    const int L = resolve_depth(m, n, k, cutoff, variant, 4);
    const long long unit = 256LL << L;  // panel height granularity: whole 256-row tiles per block
    const int P = 4;
    const long long mp = round_up(ceil_div(m, P), unit);
    if ((cutoff > 0 || algo == SW_ALGO_NAIVE) && (algo == SW_ALGO_NAIVE || sched == SW_SCHED_FUSED) &&
        n >= 1024 && k >= 1024 && m >= 2 * mp && (long long)m * n + (long long)k * n + (long long)m * k >= (16LL << 20))
        return host_panels(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, L, (int)mp, dA, lda2, dB, ldb2, dC,
                           ldc2, s);
    if (m && k) e = cudaMemcpy2DAsync(dA, lda2 * 4, A, (size_t)lda * 4, (size_t)k * 4, m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && k && n)
        e = cudaMemcpy2DAsync(dB, ldb2 * 4, B, (size_t)ldb * 4, (size_t)n * 4, k, cudaMemcpyHostToDevice, s);
    // synchronous call: a failure returns only after the copies already queued have finished
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_fail(h, e, "host to device copy");
    }
    sw_status st = sw_smm(h, dA, (int)lda2, dB, (int)ldb2, dC, (int)ldc2, m, n, k, cutoff, variant, stream);
    if (st != SW_OK) {
        cudaStreamSynchronize(s);
        return st;
    }
    if (m && n) e = cudaMemcpy2DAsync(C, (size_t)ldc * 4, dC, ldc2 * 4, (size_t)n * 4, m, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_fail(h, e, "device to host copy");
    }
    return sw_sync(h, stream);
}

sw_status sw_sync(sw_handle h, void* stream) {
    if (!h) return SW_EINVAL;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int code = 0;
    e = cudaMemcpy(&code, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word read");
    if (code != 0) {
        cudaMemset(h->d_err, 0, sizeof(int));
        {   // an aborted launch leaves ordering counters out of step: rebuild every plan
            std::lock_guard<std::mutex> lock(h->mu);
            flush_plans(h);
        }
        if (code == ERR_ALIGN) return fail(h, SW_ECUDA, "kernel rejected a misaligned TMA coordinate");
        return fail(h, SW_ETIMEOUT, "bounded device wait expired (code " + std::to_string(code) + ")");
    }
    return SW_OK;
}

sw_status sw_selftest_expired_wait(sw_handle h, void* stream) {
    if (!h) return SW_EINVAL;
    cudaSetDevice(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = 256;  // one 256-wide tile column, two 128-row tiles
    const size_t mat = (size_t)n * n * sizeof(float);
    // device block: A | B | C | tensor map of C | leaf | target | epoch, finished-CTA count, 2 counters
    const size_t o_map = 3 * mat, o_leaf = o_map + sizeof(CUtensorMap), o_tgt = o_leaf + sizeof(Leaf),
                 o_flags = round_up((long long)(o_tgt + sizeof(Target)), 64), total = o_flags + 4 * sizeof(unsigned);
    char* d = nullptr;
    if (cudaMalloc(&d, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SW_ENOMEM, "self-test buffers");
    }
    MapSet maps;
    memset(&maps, 0, sizeof(maps));
    CUtensorMap cmap;
    float* A = reinterpret_cast<float*>(d);
    float* B = reinterpret_cast<float*>(d + mat);
    float* C = reinterpret_cast<float*>(d + 2 * mat);
    if (!make_map_f32(&maps.m[0], A, n, n, n, 32, tf32_tile_m()) || !make_map_f32_n(&maps.m[1], B, n, n, n) ||
        !make_map_f32(&cmap, C, n, n, n, 32, 32)) {
        cudaFree(d);
        return fail(h, SW_ECUDA, "self-test tensor maps");
    }
    Leaf lf;
    memset(&lf, 0, sizeof(lf));
    lf.tag = -1;
    lf.a_map = 0;
    lf.b_map = 1;
    lf.m = n;
    lf.n = n;
    lf.kblocks = n / tf32_tile_k();
    lf.tiles_n = 1;
    lf.tgt_count = 1;
    Target t;
    memset(&t, 0, sizeof(t));
    t.c = C;
    t.ldc = n;
    t.rows = t.cols = n;
    t.sign = 1.f;
    t.mode = TGT_ATOMIC;  // ordered after a first write that no leaf of the launch makes
    t.vec_ok = 1;
    t.map = 0;
    t.flag_base = 0;
    t.flag_cols = 1;
    cudaError_t e = cudaMemsetAsync(d, 0, total, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_map, &cmap, sizeof(cmap), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_leaf, &lf, sizeof(lf), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + o_tgt, &t, sizeof(t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_gemm_tf32n(256, maps, nullptr, reinterpret_cast<const Leaf*>(d + o_leaf), 1,
                              reinterpret_cast<const Target*>(d + o_tgt), reinterpret_cast<const CUtensorMap*>(d + o_map),
                              reinterpret_cast<unsigned*>(d + o_flags), 2, h->d_err, h->sms, s, false);
    sw_status st = e == cudaSuccess ? sw_sync(h, stream) : cuda_fail(h, e, "self-test launch");
    cudaStreamSynchronize(s);
    cudaFree(d);
    return st;
}

sw_status sw_profile(sw_handle h, int enable) {
    if (!h) return SW_EINVAL;
    std::lock_guard<std::mutex> lock(h->mu);
    h->prof = enable != 0;
    return SW_OK;
}

sw_status sw_profile_read(sw_handle h, int nkinds, int* launches, double* ms) {
    if (!h || nkinds < 0 || (nkinds > 0 && (!launches || !ms))) return SW_EINVAL;
    std::lock_guard<std::mutex> lock(h->mu);
    for (int i = 0; i < nkinds; ++i) { launches[i] = 0; ms[i] = 0.0; }
    cudaError_t err = cudaSuccess;
    for (auto& r : h->prof_live) {
        cudaError_t e = cudaEventSynchronize(r.e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.e0, r.e1);
        if (e != cudaSuccess) err = e;
        if (r.kind >= 0 && r.kind < nkinds) { launches[r.kind] += 1; ms[r.kind] += t; }
        h->prof_free.push_back(r.e0);
        h->prof_free.push_back(r.e1);
    }
    h->prof_live.clear();
    if (err != cudaSuccess) return cuda_fail(h, err, "profile read");
    return SW_OK;
}

sw_status sw_error_norms(sw_handle h, int eb, int m, int n, int k, const void* A, int lda, const void* B, int ldb,
                         const void* C, int ldc, const double* R, int ldr, double* out, void* stream) {
    if (!h || !out || (eb != 4 && eb != 8) || m < 0 || n < 0 || k < 0) return fail(h, SW_EINVAL, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemsetAsync(h->d_norms, 0, 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = launch_norms(eb, m, n, k, A, lda, B, ldb, C, ldc, R, ldr, h->d_norms, s);
    unsigned long long bits[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, h->d_norms, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "norms");
    for (int i = 0; i < 3; ++i) memcpy(&out[i], &bits[i], sizeof(double));
    return SW_OK;
}

static sw_status server_fail(sw_handle h, sw_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(h->mu);
    h->last_error = msg;
    return st;
}

sw_status sw_server_start(sw_handle h, const sw_server_cfg* cfg) {
    if (!h) return SW_EINVAL;
    if (h->server) return server_fail(h, SW_EINVAL, "serving loop already started");
    if (cfg && (cfg->sm_share < 0 || cfg->max_inflight < 0 || cfg->idle_us < 0))
        return server_fail(h, SW_EINVAL, "negative serving parameter");
    cudaSetDevice(h->device);
    Server* s = new Server();
    std::string msg;
    const sw_status st = s->init(h, cfg, &msg);
    if (st != SW_OK) {
        delete s;
        return server_fail(h, st, msg);
    }
    s->thr = std::thread(&Server::loop, s);
    h->server = s;
    return SW_OK;
}

sw_status sw_server_submit(sw_handle h, const sw_request* q, uint64_t* ticket) {
    if (!h || !q || !ticket) return SW_EINVAL;
    Server* s = h->server;
    if (!s) return server_fail(h, SW_EINVAL, "serving loop not started");
    const int m = q->m, n = q->n, k = q->k;
    if (q->elem_bytes != 4 && q->elem_bytes != 8) return server_fail(h, SW_EINVAL, "elem_bytes must be 4 or 8");
    if (m < 0 || n < 0 || k < 0) return server_fail(h, SW_EINVAL, "negative dimension");
    if ((m && k && !q->A) || (k && n && !q->B) || (m && n && !q->C))
        return server_fail(h, SW_EINVAL, "null matrix pointer");
    if ((m && k && q->lda < std::max(k, 1)) || (k && n && q->ldb < std::max(n, 1)) ||
        (m && n && q->ldc < std::max(n, 1)))
        return server_fail(h, SW_EINVAL, "leading dimension smaller than the row length");
    // size the workspace on the caller's thread (planning only; no device work)
    sw_handle_s tmp;
    Plan dryp;
    char* base = reinterpret_cast<char*>(static_cast<uintptr_t>(1) << 20);
    sw_status st = build_plan(&tmp, q->elem_bytes, q->A, q->lda, q->B, q->ldb, q->C, q->ldc, m, n, k, q->cutoff,
                              q->variant, true, &dryp, base, true);
    if (st != SW_OK) return server_fail(h, st, tmp.last_error);
    const size_t need = (size_t)round_up((long long)dryp.ws_need, (long long)SRV_ALIGN);
    if (need > s->arena.bytes)
        return server_fail(h, SW_EBUDGET, "request workspace " + std::to_string(need) + " B exceeds the serving arena " +
                                              std::to_string(s->arena.bytes) + " B");
    ServerReq* r = new ServerReq();
    r->req = *q;
    r->need = need;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->dead != SW_OK) {
            const sw_status d = s->dead;
            const std::string msg = s->dead_msg;
            delete r;
            return server_fail(h, d, msg);
        }
        if (s->quit) { delete r; return server_fail(h, SW_EINVAL, "serving loop is stopping"); }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return SW_OK;
}

sw_status sw_server_wait(sw_handle h, uint64_t ticket, int64_t timeout_ns) {
    if (!h) return SW_EINVAL;
    Server* s = h->server;
    if (!s) return server_fail(h, SW_EINVAL, "serving loop not started");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        lk.unlock();
        return server_fail(h, SW_EINVAL, "unknown ticket (never issued, or already collected)");
    }
    ServerReq* r = it->second;
    auto done = [r] { return r->state == RQ_DONE; };
    if (timeout_ns < 0) {
        s->cv_done.wait(lk, done);
    } else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done)) {
        lk.unlock();
        return server_fail(h, SW_ETIMEOUT, "request not complete within the timeout");
    }
    const sw_status st = r->status;
    const std::string msg = r->msg;
    s->reqs.erase(it);
    delete r;
    lk.unlock();
    if (st != SW_OK) return server_fail(h, st, msg);
    return SW_OK;
}

sw_status sw_server_stop(sw_handle h) {
    if (!h) return SW_EINVAL;
    Server* s = h->server;
    if (!s) return server_fail(h, SW_EINVAL, "serving loop not started");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
    }
    s->cv_work.notify_all();
    s->thr.join();  // drains: every submitted request completes first
    s->release_device();
    for (auto& kv : s->reqs) delete kv.second;
    s->reqs.clear();
    h->server = nullptr;
    delete s;
    return SW_OK;
}

}  // extern "C"
