// runtime.cu -- the handle's workspace, plan execution (eager or through a captured CUDA graph),
// the plan cache, the autotuner (cutoff <= 0), single and batched products, and the host-operand
// row-panel pipeline.
#include <cstdlib>
#include <cstring>

#include "host.h"

namespace swh {

cudaEvent_t prof_event(sw_handle h) {
    if (!h->prof_free.empty()) {
        cudaEvent_t e = h->prof_free.back();
        h->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

sw_status fail(sw_handle h, sw_status s, const std::string& msg) {
    if (h) h->last_error = msg;
    return s;
}

sw_status cuda_fail(sw_handle h, cudaError_t e, const char* where) {
    return fail(h, SW_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void flush_plans(sw_handle h) {
    if (h->plans.empty()) return;
    cudaDeviceSynchronize();
    for (auto& kv : h->plans) delete kv.second;
    h->plans.clear();
}

// Make the workspace at least `need` bytes (flushes cached plans, which point into it).
sw_status ensure_ws(sw_handle h, size_t need) {
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

sw_status run_ops(sw_handle h, Plan* plan, cudaStream_t s, size_t first, size_t last) {
    char* blob = static_cast<char*>(plan->d_blob);
    for (size_t oi = first; oi < last && oi < plan->ops.size(); ++oi) {
        Op& o = plan->ops[oi];
        cudaError_t e = cudaSuccess;
        // (a paired block addition is profiled as a block addition)
        sw_handle_s::ProfRec rec = {o.kind == OP_ADDSUB2 ? (int)OP_ADDSUB : (int)o.kind, nullptr, nullptr};
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
                if (o.pack)
                    e = launch_gemm_tf32n_pack(gm, lv, o.nleaves, tv, tm, fl, o.items, h->d_err, h->sms, s, il,
                                               reinterpret_cast<const CopyJob*>(blob + o.jobs_off), o.njobs, o.tiles);
                else
                    e = o.nmaj ? launch_gemm_tf32n(o.bn, o.maps, gm, lv, o.nleaves, tv, tm, fl, o.items, h->d_err,
                                                   h->sms, s, o.pair, il, it, o.units)
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
            case OP_ADDSUB2:
                e = launch_addsub2(o.eb, o.job_a, o.job_b, s);
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

sw_status run_plan(sw_handle h, Plan* plan, cudaStream_t s) {
    return run_ops(h, plan, s, 0, plan->ops.size());
}

// Run a plan: eagerly, or (batched plans, profiling off) through its captured CUDA graph.
sw_status execute(sw_handle h, Plan* plan, cudaStream_t s) {
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

// Plan construction: a dry run sizes the workspace, the real run fills the plan, whose descriptors
// are uploaded once.  Growing the workspace flushes cached plans, so callers size every plan they
// will hold before building any of them.

sw_status plan_need(const PlanBuilder& build, size_t* need) {
    Plan d;
    sw_status st = build(true, &d);
    if (st == SW_OK) *need = d.ws_need;
    return st;
}

sw_status plan_make(sw_handle h, const PlanBuilder& build, Plan** out) {
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

void plan_cache(sw_handle h, const std::string& key, Plan* plan) {
    if (h->plans.size() >= 256) flush_plans(h);
    h->plans[key] = plan;
}

sw_status cached_plan(sw_handle h, const std::string& key, const PlanBuilder& build, Plan** out) {
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
sw_status time_plan(sw_handle h, Plan* plan, cudaStream_t s, double* ms) {
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
sw_status tune(sw_handle h, const std::string& key, const std::vector<PlanBuilder>& cands, cudaStream_t s,
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

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

sw_status do_mm(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int m,
                       int n, int k, int cutoff, uint32_t variant, void* stream, uint32_t top_mask, int b_sums_mode,
                       char* b_sums) {
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
            return build_plan(h, eb, A, lda, B, ldb, C, ldc, m, n, k, c, variant, dry, p, nullptr, false, top_mask,
                              b_sums_mode, b_sums);
        });
    };
    auto key_of = [&](int c) {
        char key[256];
        snprintf(key, sizeof(key), "%d|%p|%d|%p|%d|%p|%d|%d|%d|%d|%d|%u|%x|%d|%p", eb, A, lda, B, ldb, C, ldc, m, n, k,
                 c, variant, top_mask, b_sums_mode, (void*)b_sums);
        return std::string(key);
    };
    // cutoff <= 0: the autotuner picks the depth on the first call for this shape and variant (not
    // under stream capture, and not for IN_PLACE, whose runs overwrite A and B)
    const uint32_t algo = variant & SW_ALGO_MASK, sched = variant & SW_SCHED_MASK;
    if (cutoff <= 0 && algo != SW_ALGO_NAIVE && sched != SW_SCHED_IN_PLACE && top_mask == 0x7Fu && b_sums_mode == 0 &&
        !capturing(s) && m && n && k) {
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

// sw_mm_batched after argument checks: plan key, autotuned tile shape and cutoff, graph replay.
sw_status do_batched(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant, void* stream) {
    std::lock_guard<std::mutex> lock(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // plan key: the problem list's bytes
    std::string key = "B|" + std::to_string(count) + "|" + std::to_string(cutoff) + "|" + std::to_string(variant) + "|";
    key.append(reinterpret_cast<const char*>(probs), sizeof(sw_problem) * (size_t)count);
    struct Cfg { int bn, pair, cutoff; };  // pair 2: CTA pairs packing operands inside the GEMM launch
    auto builder = [=](Cfg c) {
        return PlanBuilder([=](bool dry, Plan* p) {
            return build_batched_plan(h, count, probs, c.cutoff, variant, dry, p, c.bn, c.pair != 0, c.pair == 2);
        });
    };
    auto key_of = [&](Cfg c) {
        return key + "|" + std::to_string(c.bn) + "|" + std::to_string(c.pair) + "|" + std::to_string(c.cutoff);
    };
    // a given cutoff: CTA pairs, packing inside the GEMM launch where no product recurses (the
    // autotuner's pick on the uneven 512-product workload); SWMM_BATCH_FORM = cta | pair | pack
    // selects a form (diagnostics and tests)
    static const int form = [] {
        const char* e = getenv("SWMM_BATCH_FORM");
        return !e ? 2 : !strcmp(e, "cta") ? 0 : !strcmp(e, "pair") ? 1 : 2;
    }();
    Cfg cfg = {256, tf32_bt_form() ? 0 : form, cutoff};
    // cutoff <= 0: the autotuner times the grouped launch's tile shape (128- or 256-wide tiles on one
    // CTA, 256 x 256 tiles on CTA pairs, with the packing copies before the GEMM launch or inside it)
    // and the recursion cutoff on this problem list, once
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
                cs.push_back({256, 2, none});
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

// Host-operand product in row panels of height mp (the last one lower): B goes over first, then
// panel i of A on the copy-in stream; panel i of C = A_i B runs on the caller's stream at the
// whole product's depth L (the panel's cutoff is its own smallest block side at depth L, which
// gives exactly L levels while that side is >= 2); panel i of C comes back on the copy-out stream
// while later panels still arrive and compute.  Row panels keep every copy one contiguous run.
sw_status host_panels(sw_handle h, const float* A, int lda, const float* B, int ldb, float* C, int ldc, int m,
                             int n, int k, int cutoff, uint32_t variant, int L, int mp, float* dA, long long lda2,
                             float* dB, long long ldb2, float* dC, long long ldc2, char* dS, cudaStream_t s) {
    const int npan = (int)ceil_div(m, mp);
    {
        std::lock_guard<std::mutex> lock(h->mu);
        cudaSetDevice(h->device);
        if (!h->io_in && cudaStreamCreateWithFlags(&h->io_in, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "copy stream");
        if (!h->io_out && cudaStreamCreateWithFlags(&h->io_out, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "copy stream");
        while ((int)h->io_ev.size() < 2 * npan + 3) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
                return cuda_fail(h, cudaGetLastError(), "copy event");
            h->io_ev.push_back(ev);
        }
    }
    // [0] start, [1 + i] A_i arrived, [1 + npan + i] C_i done, [1 + 2 npan] out done, [2 + 2 npan] B arrived
    cudaEvent_t* ev = h->io_ev.data();
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
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + 2 * npan], h->io_in);
    for (int i = 0; i < npan && e == cudaSuccess; ++i) {
        const int r0 = i * mp, hgt = std::min(mp, m - r0);
        e = cudaMemcpy2DAsync(dA + r0 * lda2, lda2 * 4, A + (size_t)r0 * lda, (size_t)lda * 4, (size_t)k * 4, hgt,
                              cudaMemcpyHostToDevice, h->io_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + i], h->io_in);
    }
    if (e != cudaSuccess) return drained(cuda_fail(h, e, "host to device copy"));
    // B's operand sums once for all panels at the whole product's depth, as soon as B has arrived
    const int cut_l = (int)std::min(std::min(ceil_div(mp, 1LL << L), ceil_div(n, 1LL << L)), ceil_div(k, 1LL << L));
    if (dS && (cut_l < 2 || resolve_depth(std::min(mp, m), n, k, cut_l, variant, 4) != L)) dS = nullptr;
    if (dS) {
        e = cudaStreamWaitEvent(s, ev[2 + 2 * npan], 0);
        if (e != cudaSuccess) return drained(cuda_fail(h, e, "panel order"));
        sw_status st = do_mm(h, 4, dA, (int)lda2, dB, (int)ldb2, dC, (int)ldc2, std::min(mp, m), n, k, cut_l, variant, s,
                             0x7Fu, 1, dS);
        if (st != SW_OK) return drained(st);
    }
    for (int i = 0; i < npan; ++i) {
        const int r0 = i * mp, hgt = std::min(mp, m - r0);
        e = cudaStreamWaitEvent(s, ev[1 + i], 0);
        if (e != cudaSuccess) return drained(cuda_fail(h, e, "panel order"));
        int cut = cutoff;
        bool shared = false;  // this panel reads the shared B-side sums
        if ((variant & SW_ALGO_MASK) != SW_ALGO_NAIVE) {
            const long long d = 1LL << L;
            cut = (int)std::min(std::min(ceil_div(hgt, d), ceil_div(n, d)), ceil_div(k, d));
            if (cut < 2 || resolve_depth(hgt, n, k, cut, variant, 4) != L) cut = cutoff;  // low last panel
            else shared = dS != nullptr;
        }
        sw_status st = do_mm(h, 4, dA + r0 * lda2, (int)lda2, dB, (int)ldb2, dC + r0 * ldc2, (int)ldc2, hgt, n, k, cut,
                             variant, s, 0x7Fu, shared ? 2 : 0, shared ? dS : nullptr);
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

}  // namespace swh
