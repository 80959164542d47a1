// server.cu -- the serving loop (sw_server_*): continuous batching of submitted products on a
// device-resident persistent GEMM and side streams.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "host.h"
#include "arena.h"

using namespace swh;

// ====================================================================== serving loop
// A host thread admits submitted requests in arrival order while their workspace fits the arena
// and a completion slot is free.  Each admitted request is planned inside the arena.  When the
// plan ends in a grouped TF32 GEMM (BN 256, no ordering counters), every op before it runs on a
// side stream, and the GEMM's leaves, targets and tensor maps are appended to the descriptor
// arrays of the resident kernel, which claims the published tiles one by one on its share of the
// SMs; the request is complete when its counter reaches 4 per tile (one per epilogue warp).
// Other plans (FP64, split-BF16 leaves, padded or peeled shapes) run whole on a side stream with
// the SMs the resident kernel leaves free.  When the descriptor arrays are full the kernel is asked
// to exit once it has claimed every published tile, and a new generation starts after it has; the
// host thread never waits for that (the kernel may be queued behind long side-stream blocks), so
// other requests keep starting and completing meanwhile.
namespace {

constexpr int SRV_SIDE = 4;                   // side streams: [0, SRV_SIDE / 2) high priority, the rest low
// A request whose work is estimated below this many milliseconds (TF32 leaves at ~900 TFLOP/s, FP64
// at ~1.5 TFLOP/s) runs on a high-priority side stream, so that its blocks take the SMs before
// pending blocks of long requests (the FP64 n = 8192 products take half a second each).
constexpr double SRV_SHORT_MS = 2.0;
constexpr unsigned SRV_MAX_ITEMS = 1u << 21;  // published tiles per generation
constexpr int SRV_MAX_LEAVES = 1 << 16;
constexpr int SRV_MAX_TARGETS = 1 << 18;
constexpr int SRV_MAX_MAPS = 1 << 14;   // operand tensor maps
constexpr int SRV_MAX_TMAPS = 1 << 16;  // target tensor maps
constexpr size_t SRV_BLOB_BYTES = 256u << 20;
constexpr size_t SRV_ALIGN = 1024;

// RQ_LAUNCH: planned, its ops being enqueued by the launcher thread; RQ_LFAIL: that failed.
enum ReqState { RQ_QUEUED = 0, RQ_PRE = 1, RQ_PUBLISHED = 2, RQ_DONE = 3, RQ_LAUNCH = 4, RQ_LFAIL = 5 };

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
    cudaStream_t stream = nullptr;  // its side stream
    sw_status status = SW_OK;
    std::string msg;
    sw_status launch_status = SW_OK;  // set by the launcher thread
    std::string launch_msg;
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
    // Long requests' ops are enqueued by a launcher thread: a deep FP64 plan holds thousands of
    // kernels, a launch into a full stream queue blocks until the GPU drains it, and this thread
    // must keep starting and completing the other requests meanwhile.
    sw_handle_s shadow_l;  // the launcher's copy of `shadow`
    std::thread launcher;
    std::mutex lmu;  // guards lq, lquit, lbusy
    std::condition_variable lcv, lcv_idle;
    std::deque<ServerReq*> lq;
    bool lquit = false;
    int lbusy = 0;
    void launch_loop();
    void launcher_drop_and_wait();
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
    int side_rr[2] = {0, 0};  // round robin within the high- / low-priority side streams
    unsigned n_items = 0;
    int n_leaves = 0, n_targets = 0, n_maps = 0, n_tmaps = 0;
    bool res_launched = false;
    bool stopping = false;  // the resident kernel was asked to exit (a new generation follows)
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
    shadow_l.device = device;
    shadow_l.sms = shadow.sms;
    shadow_l.d_err = shadow.d_err;
    if (cudaHostAlloc(&poll_h, ctl_bytes(), cudaHostAllocDefault) != cudaSuccess) return oom("the poll buffer");
    if (cudaHostAlloc(&mapped_h, 256, cudaHostAllocMapped) != cudaSuccess) return oom("the mapped words");
    memset(mapped_h, 0, 256);
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&mapped_d), mapped_h, 0) != cudaSuccess)
        return oom("the mapped words (device view)");
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) return oom("stream priorities");
    // the resident kernel's CTAs take SMs ahead of pending blocks of long side-stream work
    if (cudaStreamCreateWithPriority(&res_stream, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctl_stream, cudaStreamNonBlocking) != cudaSuccess)
        return oom("streams");
    for (int i = 0; i < SRV_SIDE; ++i)
        if (cudaStreamCreateWithPriority(&side[i], cudaStreamNonBlocking, i < SRV_SIDE / 2 ? prio_high : prio_low) !=
            cudaSuccess)
            return oom("streams");
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
    launcher_drop_and_wait();  // requests it had not launched are completed below with the rest
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
    ResidentCtl c = {};
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
    const double work_ms = 2.0 * (double)q.m * q.n * q.k / (q.elem_bytes == 8 ? 1.5e9 : 9e11);
    const int cls = work_ms < SRV_SHORT_MS ? 0 : 1;
    cudaStream_t s = side[cls * (SRV_SIDE / 2) + side_rr[cls]];
    side_rr[cls] = (side_rr[cls] + 1) % (SRV_SIDE / 2);
    r->stream = s;
    if (!r->plan.blob.empty()) {
        const size_t nb = (size_t)round_up((long long)r->plan.blob.size(), 256);
        size_t off = 0;
        if (!blobs.alloc(nb, &off)) { complete(r, SW_EBUDGET, "serving: descriptor pool full"); return; }
        r->blob_off = off;
        r->blob_bytes = nb;
        r->plan.d_blob = blob_mem + off;
    }
    r->resident = resident_form(r->plan);
    r->ev = take_event();
    if (cls == 1) {  // long: the launcher thread enqueues it
        {
            std::lock_guard<std::mutex> lk(mu);
            r->state = RQ_LAUNCH;
        }
        {
            std::lock_guard<std::mutex> lk(lmu);
            lq.push_back(r);
        }
        lcv.notify_one();
        return;
    }
    if (r->blob_bytes)
        cudaMemcpyAsync(r->plan.d_blob, r->plan.blob.data(), r->plan.blob.size(), cudaMemcpyHostToDevice, s);
    st = run_ops(&shadow, &r->plan, s, 0, r->plan.ops.size() - (r->resident ? 1 : 0));
    if (st != SW_OK) {
        cudaStreamSynchronize(s);
        complete(r, st, shadow.last_error);
        return;
    }
    cudaEventRecord(r->ev, s);
    std::lock_guard<std::mutex> lk(mu);
    r->state = RQ_PRE;
}

// The launcher thread: enqueue a long request's ops (all but a resident GEMM) on its side stream,
// record its event and hand it back in RQ_PRE (RQ_LFAIL if a launch failed).
void Server::launch_loop() {
    cudaSetDevice(device);
    for (;;) {
        ServerReq* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(lmu);
            lcv.wait(lk, [&] { return lquit || !lq.empty(); });
            if (lq.empty()) break;
            r = lq.front();
            lq.pop_front();
            ++lbusy;
        }
        if (r->blob_bytes)
            cudaMemcpyAsync(r->plan.d_blob, r->plan.blob.data(), r->plan.blob.size(), cudaMemcpyHostToDevice,
                            r->stream);
        shadow_l.last_error.clear();
        const sw_status st = run_ops(&shadow_l, &r->plan, r->stream, 0, r->plan.ops.size() - (r->resident ? 1 : 0));
        if (st != SW_OK) cudaStreamSynchronize(r->stream);
        else cudaEventRecord(r->ev, r->stream);
        {
            std::lock_guard<std::mutex> lk(mu);
            r->launch_status = st;
            r->launch_msg = shadow_l.last_error;
            r->state = st == SW_OK ? RQ_PRE : RQ_LFAIL;
        }
        {
            std::lock_guard<std::mutex> lk(lmu);
            --lbusy;
        }
        lcv_idle.notify_all();
    }
}

// Drop the requests still waiting for the launcher (they stay in `active`, never launched) and
// wait until the launcher is idle.
void Server::launcher_drop_and_wait() {
    std::unique_lock<std::mutex> lk(lmu);
    lq.clear();
    lcv_idle.wait(lk, [&] { return lbusy == 0; });
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
    std::vector<ServerReq*> pre, ready, published, lfail;
    {
        std::lock_guard<std::mutex> lk(mu);  // the launcher thread moves requests out of RQ_LAUNCH
        for (ServerReq* r : active) {
            if (r->state == RQ_PRE) pre.push_back(r);
            else if (r->state == RQ_PUBLISHED) published.push_back(r);
            else if (r->state == RQ_LFAIL) lfail.push_back(r);
        }
    }
    for (ServerReq* r : lfail) complete(r, r->launch_status, r->launch_msg);
    for (ServerReq* r : pre) {
        const cudaError_t e = cudaEventQuery(r->ev);
        if (e == cudaSuccess) ready.push_back(r);
        else if (e != cudaErrorNotReady) { fatal(std::string("serving: ") + cudaGetErrorString(e)); return true; }
    }
    if (ready.empty() && published.empty()) return !lfail.empty();
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
        if (stopping) {  // the kernel may already have stopped claiming: wait for the next generation
            deferred = true;
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
    {
        std::lock_guard<std::mutex> lk(mu);
        for (ServerReq* r : active) pending |= r->state == RQ_PUBLISHED;
    }
    if (stopping && !kernel_running()) {  // the old generation's kernel has exited
        set_mapped(32, 0u);
        stopping = false;
        moved = true;
    }
    if (stopping) {
        // its claimed tiles finish and report; requests keep starting meanwhile (no host wait:
        // the kernel may still be queued behind long side-stream work)
    } else if (pending) {
        if (!kernel_running()) {
            if (launch_resident() != SW_OK) { fatal("serving: resident kernel launch failed"); return true; }
            moved = true;
        }
    } else if (n_items > 0 && (deferred || !kernel_running())) {
        if (kernel_running()) {
            set_mapped(32, 1u);  // exit once every published tile is claimed; reset when it has
            stopping = true;
        } else {
            reset_generation();
        }
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

static sw_status server_fail(sw_handle h, sw_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(h->mu);
    h->last_error = msg;
    return st;
}

extern "C" {

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
    s->launcher = std::thread(&Server::launch_loop, s);
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
    {
        std::lock_guard<std::mutex> lk(s->lmu);
        s->lquit = true;
    }
    s->lcv.notify_all();
    s->launcher.join();
    s->release_device();
    for (auto& kv : s->reqs) delete kv.second;
    s->reqs.clear();
    h->server = nullptr;
    delete s;
    return SW_OK;
}

}  // extern "C"
