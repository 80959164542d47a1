// host.h -- host-side internals shared by the planner (planner.cu, fused.cu), the runtime
// (runtime.cu), the serving loop (server.cu) and the C ABI (api.cu): the op list a plan lowers a
// product to, the handle, and the functions that build, cache, tune and run plans.
#pragma once

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

#include <set>
#include <tuple>

#include "../../include/swmm.h"
#include "internal.h"
#include "plan.h"

namespace swh {
using namespace swk;

// ------------------------------------------------------------------ tensor maps, switches (planner.cu)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable)
EncodeTiledFn encode_fn();
// FP32 row-major view rows x cols (ld elements) -> 2-D tensor map with a box of box_cols (innermost,
// 128 bytes) x box_rows, 128-byte swizzle, zero fill out of bounds.
bool make_map_f32(CUtensorMap* m, const void* base, int rows, int cols, long long ld, int box_cols, int box_rows);
// FP32 row-major k x n view of an N-major B operand -> 32 x 32 boxes, 128-byte swizzle with 32-byte atoms.
bool make_map_f32_n(CUtensorMap* m, const void* base, int rows, int cols, long long ld);
// BF16 row-major view (ld a multiple of 8) -> 64-column x box_rows boxes, 128-byte swizzle.
bool make_map_bf16(CUtensorMap* m, const void* base, int rows, int cols, long long ld, int box_rows);
inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }
inline long long ceil_div(long long x, long long a) { return (x + a - 1) / a; }
// SWMM_TF32_BT=1: TF32 leaves read B as B^T (diagnostics); SWMM_TF32_BN: forced tile width (0: none)
bool tf32_bt_form();
int bn_override();

// ------------------------------------------------------------------ plan
enum OpKind {
    OP_GEMM_TF32, OP_GEMM_SIMT, OP_ADDSUB, OP_COPY_PAD, OP_PREADD, OP_MEMSET, OP_TRANSPOSE, OP_TRANSPOSE_SQ,
    OP_SPLIT, OP_GEMM_BF16X3, OP_BATCH_COPY, OP_SPLIT_TF32, OP_GEMM_TF32X3, OP_PREADD_SPLIT, OP_ADDSUB2
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
    bool pack = false;           // batched TF32N pair GEMM that also runs the pack jobs at jobs_off
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
    AddJob job_a, job_b;    // OP_ADDSUB2: two block additions in one launch
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

// Elements of the B-side operand sums of a FUSED FP32 product with TF32 leaves at depth L (fused.cu).
long long fused_b_sum_elems(int algo, int k, int n, int L);
// Recursion depth of a product (the Sec. 3.4 cutoff rule, capped for the FUSED schedule).
int resolve_depth(int m, int n, int k, int cutoff, uint32_t variant, int eb);

}  // namespace swh

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
    std::unordered_map<std::string, swh::Plan*> plans;
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

namespace swh {

// ------------------------------------------------------------------ runtime (runtime.cu)
sw_status fail(sw_handle h, sw_status s, const std::string& msg);
sw_status cuda_fail(sw_handle h, cudaError_t e, const char* where);
// Free every cached plan (waits for the device first).
void flush_plans(sw_handle h);
// Make the workspace at least `need` bytes (flushes cached plans, which point into it).
sw_status ensure_ws(sw_handle h, size_t need);
// Build the whole plan for one product (planner.cu); server: plan inside a region of the serving arena
sw_status build_plan(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int m,
                     int n, int k, int cutoff, uint32_t variant, bool dry, Plan* plan, char* ws_base = nullptr,
                     bool server = false, uint32_t top_mask = 0x7Fu, int b_sums_mode = 0,
                     char* b_sums = nullptr);
// Plan of a batch of FP32 products in one grouped launch (planner.cu)
sw_status build_batched_plan(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant, bool dry,
                             Plan* plan, int bn = 256, bool pair = false, bool pack = false);
// Launch ops [first, last) of a plan on `s`.
sw_status run_ops(sw_handle h, Plan* plan, cudaStream_t s, size_t first, size_t last);
sw_status run_plan(sw_handle h, Plan* plan, cudaStream_t s);
// Run a plan eagerly, or (batched plans, profiling off) through its captured CUDA graph.
sw_status execute(sw_handle h, Plan* plan, cudaStream_t s);
using PlanBuilder = std::function<sw_status(bool dry, Plan* plan)>;
sw_status plan_need(const PlanBuilder& build, size_t* need);
sw_status plan_make(sw_handle h, const PlanBuilder& build, Plan** out);
void plan_cache(sw_handle h, const std::string& key, Plan* plan);
sw_status cached_plan(sw_handle h, const std::string& key, const PlanBuilder& build, Plan** out);
sw_status time_plan(sw_handle h, Plan* plan, cudaStream_t s, double* ms);
sw_status tune(sw_handle h, const std::string& key, const std::vector<PlanBuilder>& cands, cudaStream_t s, int* best,
               double* best_ms);
bool capturing(cudaStream_t s);
// One product through the plan cache (and the autotuner for cutoff <= 0): sw_smm / sw_dmm; with
// top_mask != 0x7F only the contributions of those top-level products (sw_mm_products, no tuning).
sw_status do_mm(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int m, int n,
                int k, int cutoff, uint32_t variant, void* stream, uint32_t top_mask = 0x7Fu, int b_sums_mode = 0,
                char* b_sums = nullptr);
// A validated batch of products: sw_mm_batched.
sw_status do_batched(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant, void* stream);
// Host-operand product in row panels (sw_smm_host); dS: room for B's operand sums, computed once
// and shared by the panels (nullptr: each panel computes its own).
sw_status host_panels(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m, int n,
                      int k, int cutoff, uint32_t variant, int L, int mp, float* dA, long long lda2, float* dB,
                      long long ldb2, float* dC, long long ldc2, char* dS, cudaStream_t s);

}  // namespace swh
