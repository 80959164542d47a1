// api.cu -- the C ABI (include/swmm.h): argument checks and the calls into the runtime.  The
// planner lowers a product C <- A B into kernel launches:
//
// C <- A B into kernel launches:
//
//   NAIVE            one grouped-GEMM launch, one leaf, one STORE target (Alg. 1 on tensor cores)
//   FUSED            one operand-sum pass per operand (all L levels at once) + one grouped-GEMM
//                    launch over the 7^L leaves; the leaf epilogues add +-P into the C blocks
//   TWO_TEMP         Table 2 of Sec. 3.3, step by step, X / Y temporaries per level
//   IN_PLACE         Table 3 of Sec. 3.3, step by step, temporaries in A, B and C
//   ALLOC            Alg. 2 / Alg. 3 as written: fresh temporaries at every level
//
#include <cstring>

#include "host.h"

using namespace swh;

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

sw_status sw_mm_products(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int m,
                         int n, int k, int cutoff, uint32_t variant, uint32_t product_mask, void* stream) {
    if (!h) return SW_EINVAL;
    if (eb != 4 && eb != 8) return fail(h, SW_EINVAL, "elem_bytes must be 4 or 8");
    if ((product_mask & ~0x7Fu) != 0) return fail(h, SW_EINVAL, "product_mask has bits beyond the seven products");
    if (cutoff <= 0) cutoff = eb == 4 ? 8192 : 128;  // the static default: no tuning for partial products
    return do_mm(h, eb, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, stream, product_mask);
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
    return do_batched(h, count, probs, cutoff, variant, stream);
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

sw_status sw_smm_host(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m, int n,
                      int k, int cutoff, uint32_t variant, void* stream) {
    if (!h) return SW_EINVAL;
    if (m < 0 || n < 0 || k < 0 || (m && k && (!A || lda < k)) || (k && n && (!B || ldb < n)) ||
        (m && n && (!C || ldc < n)))
        return fail(h, SW_EINVAL, "bad host operand");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long lda2 = round_up(std::max(k, 1), 4), ldb2 = round_up(std::max(n, 1), 4), ldc2 = ldb2;
    // large FUSED / naive products with a given cutoff: A and C move in row panels so the copies
    // overlap the panel products and each other (the link is duplex)
    const uint32_t algo = variant & SW_ALGO_MASK, sched = variant & SW_SCHED_MASK;
    const int L = resolve_depth(m, n, k, cutoff, variant, 4);
    const long long unit = 256LL << L;  // panel height granularity: whole 256-row tiles per block
    const int P = 4;
    const long long mp = round_up(ceil_div(m, P), unit);
    const bool panels = (cutoff > 0 || algo == SW_ALGO_NAIVE) && (algo == SW_ALGO_NAIVE || sched == SW_SCHED_FUSED) &&
                        n >= 1024 && k >= 1024 && m >= 2 * mp &&
                        (long long)m * n + (long long)k * n + (long long)m * k >= (16LL << 20);
    // the panels share one pass of B's operand sums (FUSED, TF32 leaves read N-major)
    const bool share_b = panels && algo != SW_ALGO_NAIVE && L >= 1 && L <= 3 &&
                         (variant & SW_LEAF_MASK) == SW_LEAF_TF32 && !tf32_bt_form();
    const size_t ba = (size_t)round_up((long long)m * lda2 * 4, 256), bb = (size_t)round_up((long long)k * ldb2 * 4, 256),
                 bc = (size_t)round_up((long long)m * ldc2 * 4, 256),
                 bs = share_b ? (size_t)round_up(fused_b_sum_elems((int)algo, k, n, L) * 4, 256) : 0;
    {
        std::lock_guard<std::mutex> lock(h->mu);
        cudaSetDevice(h->device);
        if (ba + bb + bc + bs > h->io_bytes) {
            flush_plans(h);
            if (h->io) { cudaDeviceSynchronize(); cudaFree(h->io); h->io = nullptr; h->io_bytes = 0; }
            if (cudaMalloc(&h->io, ba + bb + bc + bs) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, SW_ENOMEM, "host-path buffers");
            }
            h->io_bytes = ba + bb + bc + bs;
        }
    }
    float* dA = reinterpret_cast<float*>(h->io);
    float* dB = reinterpret_cast<float*>(h->io + ba);
    float* dC = reinterpret_cast<float*>(h->io + ba + bb);
    char* dS = share_b ? h->io + ba + bb + bc : nullptr;
    cudaError_t e = cudaSuccess;
    if (panels)
        return host_panels(h, A, lda, B, ldb, C, ldc, m, n, k, cutoff, variant, L, (int)mp, dA, lda2, dB, ldb2, dC,
                           ldc2, dS, s);
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

}  // extern "C"
