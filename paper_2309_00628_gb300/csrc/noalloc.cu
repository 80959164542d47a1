// noalloc.cu -- sw_smm_noalloc: a one-level Strassen-Winograd FP32 product that never allocates
// device memory.
//
// Why it exists: some callers cannot let a library call cudaMalloc.  A serving runtime or a
// framework that reserves nearly all HBM for its own caching allocator at start-up leaves no room
// for a library allocation (it would fail or fragment the pool); a real-time or certified
// deployment may forbid any device allocation after initialisation; and code running between
// other work on a stream that must not be disturbed by an implicit synchronisation cannot take
// the cost of cudaMalloc / cudaFree.  This entry point takes the inputs and the output from the
// caller and keeps every temporary -- B^T, the operand sums S1..S4 and T1..T4, the leaf and
// target descriptors and the device error word -- in one file-scope __device__ array of fixed
// size.
//
// When the memory is taken: the array lives in this file's CUDA module, and the kernels the call
// launches live in the library's other modules.  CUDA loads modules and kernels lazily by default
// (at their first use), so the first call on a device does a one-time set-up with that device
// current: it resolves the array's device address (which loads the module and places the array
// in device memory) and loads every kernel the call launches.  From then on the array stays on
// that device until the process exits and no call takes device memory.  A caller that reserves
// the GPU's memory for itself should make its first call before reserving (or run with
// CUDA_MODULE_LOADING=EAGER, which loads everything when the context is created), and before any
// stream capture.
//
// All calls share that array and each call overwrites it.  Calls that overlap on the GPU (two
// streams, or two host threads) race on it; callers must serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/swmm.h"
#include "internal.h"
#include "plan.h"

namespace {

constexpr size_t kScratchBytes = SW_NOALLOC_SCRATCH_BYTES;  // 32 MiB
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a stand-in for the device symbol: its
// device address is obtained with cudaGetSymbolAddress below and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void noalloc_describe(swk::Leaf* leaves, swk::Target* targets, float* C, long long ldc, int m, int n,
                                 int mb, int kb, int nb, int tiles_n, int tiles_per_leaf, int vec_ok);

std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// One-time set-up of device `dev` (the current device): the scratch array's device address, the
// SM count, and every kernel the call launches loaded into device memory (so that with lazy
// module loading no later call takes device memory).  Returns nullptr on failure.
unsigned char* device_setup(int dev, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaFuncAttributes fa;
        int n = 0;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(noalloc_describe)) != cudaSuccess ||
            swk::preload_gemm_tf32() != cudaSuccess || swk::preload_transpose_preadd_f32_l1() != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return nullptr;
        }
        g_sms[dev] = n;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *sms = g_sms[dev];
    return g_scratch_ptr[dev];
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

bool map_f32(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_rows) {
    EncodeFn enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(cols > 0 ? cols : 1), (cuuint64_t)(rows > 0 ? rows : 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline long long rup(long long x, long long a) { return (x + a - 1) / a * a; }

// Scratch layout (byte offsets inside the array).
struct Layout {
    long long mb, kb, nb;                 // leaf block extents (one level)
    size_t err, leaves, targets, bt, sa, sb, total;
};

Layout layout(int m, int n, int k) {
    Layout L;
    L.mb = (m + 1) / 2;
    L.kb = rup((k + 1) / 2, 32);
    L.nb = rup((n + 1) / 2, 4);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (size_t)rup((long long)bytes, 256); return o; };
    L.err = take(256);
    L.leaves = take(7 * sizeof(swk::Leaf));
    L.targets = take(14 * sizeof(swk::Target));
    L.bt = take((size_t)n * (size_t)rup(k, 4) * 4);  // B^T, n x k
    L.sa = take((size_t)4 * L.mb * L.kb * 4);         // S1..S4 (BDPZ), dense slots
    L.sb = take((size_t)4 * L.nb * L.kb * 4);         // T1..T4, held transposed
    L.total = off;
    return L;
}

// Leaf descriptors of one Winograd level (BDPZ form, Sec. 2.3), written on the device so the
// call needs no host-to-device copy.  Leaf p = product P(p+1); its A operand is the quadrant
// A11 / A12 / A22 (map 0, in place) or a slot of the S sums (map 2), its B operand a quadrant of
// B^T (map 1) or a slot of the T sums (map 3); its targets are the C quadrants the U chain adds
// it to: C11 = P1+P2, C12 = P1+P6+P5+P3, C21 = P1+P6+P7-P4, C22 = P1+P6+P7+P5.
__global__ void noalloc_describe(swk::Leaf* leaves, swk::Target* targets, float* C, long long ldc, int m, int n,
                                 int mb, int kb, int nb, int tiles_n, int tiles_per_leaf, int vec_ok) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    // per product: A source (quadrant or -1-slot), B source in logical quadrants (or -1-slot)
    const int a_q[7] = {0, 1, -1, 3, -1, -1, -1}, a_slot[7] = {-1, -1, 3, -1, 0, 1, 2};   // S4, S1, S2, S3
    const int b_q[7] = {0, 2, 3, -1, -1, -1, -1}, b_slot[7] = {-1, -1, -1, 3, 0, 1, 2};   // T4, T1, T2, T3
    const int ntg[7] = {4, 1, 1, 1, 2, 3, 2};
    const int tq[7][4] = {{0, 1, 2, 3}, {0}, {1}, {2}, {1, 3}, {1, 2, 3}, {2, 3}};
    const float ts[7][4] = {{1, 1, 1, 1}, {1}, {1}, {-1}, {1, 1}, {1, 1, 1}, {1, 1}};
    int t = 0;
    for (int p = 0; p < 7; ++p) {
        swk::Leaf& lf = leaves[p];
        if (a_q[p] >= 0) { lf.a_map = 0; lf.a_row = (a_q[p] >> 1) * mb; lf.a_col = (a_q[p] & 1) * kb; }
        else { lf.a_map = 2; lf.a_row = a_slot[p] * mb; lf.a_col = 0; }
        // logical B quadrant (r, c) is block (c, r) of B^T
        if (b_q[p] >= 0) { lf.b_map = 1; lf.b_row = (b_q[p] & 1) * nb; lf.b_col = (b_q[p] >> 1) * kb; }
        else { lf.b_map = 3; lf.b_row = b_slot[p] * nb; lf.b_col = 0; }
        lf.m = mb;
        lf.n = nb;
        lf.kblocks = kb / 32;
        lf.tiles_n = tiles_n;
        lf.tile_begin = p * tiles_per_leaf;
        lf.tgt_begin = t;
        lf.c_row0 = 0;
        lf.c_col0 = 0;
        lf.tag = -1;
        int cnt = 0;
        for (int i = 0; i < ntg[p]; ++i) {
            const int q = tq[p][i], r = q >> 1, c = q & 1;
            const int rows = min(mb, m - r * mb), cols = min(nb, n - c * nb);
            if (rows <= 0 || cols <= 0) continue;
            swk::Target& tg = targets[t++];
            tg.c = C + (long long)r * mb * ldc + (long long)c * nb;
            tg.ldc = ldc;
            tg.rows = rows;
            tg.cols = cols;
            tg.sign = ts[p][i];
            tg.mode = swk::TGT_ATOMIC;
            tg.vec_ok = vec_ok;
            tg.map = -1;
            tg.flag_base = -1;
            tg.flag_cols = 0;
            ++cnt;
        }
        lf.tgt_count = cnt;
    }
}

}  // namespace

extern "C" sw_status sw_smm_noalloc(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m,
                                    int n, int k, void* stream) {
    if (m < 2 || n < 2 || k < 2 || !A || !B || !C || lda < k || ldb < n || ldc < n) return SW_EINVAL;
    if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15) != 0 || (lda % 4) != 0 ||
        (ldc % 4) != 0)
        return SW_EINVAL;
    const Layout L = layout(m, n, k);
    if (L.total > kScratchBytes) return SW_EBUDGET;  // the problem does not fit the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; }
    int sms = 0;
    unsigned char* base = device_setup(dev, &sms);
    if (!base) return SW_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = reinterpret_cast<int*>(base + L.err);
    swk::Leaf* leaves = reinterpret_cast<swk::Leaf*>(base + L.leaves);
    swk::Target* targets = reinterpret_cast<swk::Target*>(base + L.targets);
    float* bt = reinterpret_cast<float*>(base + L.bt);
    float* sa = reinterpret_cast<float*>(base + L.sa);
    float* sb = reinterpret_cast<float*>(base + L.sb);
    const long long ldbt = rup(k, 4);
    const int bn = L.nb <= 128 ? 128 : 256;
    const int tiles_n = (int)((L.nb + bn - 1) / bn);
    const int tiles_per_leaf = (int)((L.mb + 127) / 128) * tiles_n;

    swk::MapSet maps;
    if (!map_f32(&maps.m[0], A, m, k, lda, 128) || !map_f32(&maps.m[1], bt, n, k, ldbt, bn) ||
        !map_f32(&maps.m[2], sa, 4 * L.mb, L.kb, L.kb, 128) || !map_f32(&maps.m[3], sb, 4 * L.nb, L.kb, L.kb, bn))
        return SW_ECUDA;

    swk::PreaddArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    for (int w = 0; w < 343; ++w) pa.slot_of[w] = -1;
    pa.L = 1;
    pa.alg = 2;
    pa.out = sa;
    pa.x = A; pa.ldx = lda; pa.rows = m; pa.cols = k; pa.brows = (int)L.mb; pa.bcols = (int)L.kb;
    pa.bside = 0; pa.bt = 0;
    pa.slot_of[2] = 3; pa.slot_of[4] = 0; pa.slot_of[5] = 1; pa.slot_of[6] = 2;  // S4, S1, S2, S3
    swk::PreaddArgs pb = pa;
    pb.out = sb;
    pb.x = bt; pb.ldx = ldbt; pb.rows = n; pb.cols = k; pb.brows = (int)L.nb; pb.bcols = (int)L.kb;
    pb.bside = 1; pb.bt = 1;
    for (int w = 0; w < 343; ++w) pb.slot_of[w] = -1;
    pb.slot_of[3] = 3; pb.slot_of[4] = 0; pb.slot_of[5] = 1; pb.slot_of[6] = 2;  // T4, T1, T2, T3

    const int vec_ok = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && (ldc % 4) == 0 &&
                        ((L.nb % 4) == 0)) ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);  // the error word must start at zero
    if (e == cudaSuccess) {
        noalloc_describe<<<1, 32, 0, s>>>(leaves, targets, C, ldc, m, n, (int)L.mb, (int)L.kb, (int)L.nb, tiles_n,
                                          tiles_per_leaf, vec_ok);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = swk::launch_transpose_pad(n, k, bt, ldbt, B, ldb, k, n, s);
    if (e == cudaSuccess) e = swk::launch_preadd(4, pa, s);
    if (e == cudaSuccess) e = swk::launch_preadd(4, pb, s);
    if (e == cudaSuccess) e = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)n * 4, (size_t)m, s);  // C is summed into
    if (e == cudaSuccess)
        e = swk::launch_gemm_tf32(bn, maps, nullptr, leaves, 7, targets, nullptr, nullptr, 7 * tiles_per_leaf, err,
                                  sms, s);
    // the error word comes back on the caller's stream (no legacy-stream copy, which would wait for
    // every other blocking stream of the device)
    int code = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaGetLastError(); return SW_ECUDA; }
    return code ? SW_ETIMEOUT : SW_OK;
}
