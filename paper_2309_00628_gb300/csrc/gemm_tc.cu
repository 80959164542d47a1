// gemm_tc.cu -- grouped leaf GEMM on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
// Computes the leaf sub-products P = Aop * Bop of the recursion (Sec. 2.2 / 2.3; with a single
// leaf and a single STORE target it is the plain product of Alg. 1) and adds sign * P into
// each of the leaf's target blocks of C -- the post-additions folded into the epilogue.
//
// Operand modes:
//  * TF32N (the default TF32 form): FP32 operands staged by TMA and consumed by
//    tcgen05.mma.kind::tf32 (the tensor core reads each FP32 operand as TF32: its 10 leading
//    mantissa bits).  A K-major as stored (m x k, 128-byte swizzle); B N-major as stored (k x n):
//    32-column boxes with the 128-byte swizzle of 32-byte atoms, read by a layout-type-1
//    descriptor whose K direction comes in 4-row groups (stride 512 bytes).
//  * TF32: the same with B given as B^T (n x k), K-major (serving loop, diagnostics).
//  * BF16X3: each FP32 operand arrives split into bf16 halves hi = bf16(x), lo = bf16(x - hi);
//    per k-step the kernel issues kind::f16 MMAs hi*hi + hi*lo + lo*hi into one FP32
//    accumulator.  A K-major, B N-major (as stored, k x n).
//  * TF32X3: compensated TF32, FP32 halves hi = tf32(x), lo = x - hi; three kind::tf32 MMAs per
//    k-step (B N-major).
// Products accumulate in FP32 in tensor memory.
//
// CTA = 6 warps (10 when the launch packs operands: warps 6..9 copy them), persistent over work
// items (one item = one BM x BN output tile of one leaf):
//   warp 0      TMA producer: the A tile(s) and B tile(s) of one k-block per stage
//   warp 1      TMEM allocator + MMA issuer (one thread)
//   warps 2..5  epilogue: tcgen05.ld 32 columns at a time; each warp stages its 32 x 32 chunk
//               (with the target's sign) in 128-byte-swizzled shared memory and one lane issues a
//               TMA store (first writer) or TMA reduce-add (further contributions) per target;
//               targets without a tensor map take coalesced row stores / atomics from the same
//               staging (one 128-byte row run per warp step).
// With BN <= 256 two TMEM accumulators (2 x BN columns) let the epilogue of tile i overlap the
// MMAs of i+1.  CTA pairs (cta_group::2) take 256-row tiles; TF32N pairs also run 256 x 512 tiles
// as two N = 256 MMAs per k-step into one 512-column accumulator (fewer operand bytes per MMA,
// the epilogue no longer overlapped).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <algorithm>
#include <cstring>

#include "plan.h"
#include "ptx.cuh"
#include "internal.h"

namespace swk {

constexpr int TF_BM = 128;
constexpr int TF_BK = 32;  // TF32 k-block: 32 FP32 = 128 bytes, one swizzle row
// tiles are taken in bands of TF_GROUP_M x 128 rows, column-major inside a band: a wave of 76
// CTA pairs then covers about 12 x 6 tiles, whose A and B panels are shared by more of the wave
// than in narrower bands (DRAM re-reads fall; n = 8192 plain: 1.30 ms with 8, 1.27 ms with 24)
constexpr int TF_GROUP_M = 24;
// MODE_TF32N: TF32 with B N-major (k x n as stored): B staged in 32-column (128-byte) boxes
// with the 32-byte-atom 128-byte swizzle, read by the MMA through a layout-type-1 descriptor.
// MODE_TF32X3: compensated TF32 -- each FP32 operand arrives as (hi, lo) FP32 halves, hi = tf32(x),
// lo = x - hi; per k-step three MMAs lo*hi + hi*lo + hi*hi (A K-major, B N-major as in TF32N).
// MODE_TF32N_PACK: TF32N on CTA pairs whose launch also packs operands (batched products whose
// rows are not 16-byte aligned): four more warps per CTA copy the launch's pack jobs, tile by
// tile in job order, while the tiles of earlier products run.
constexpr int MODE_TF32 = 0, MODE_BF16X3 = 1, MODE_TF32N = 2, MODE_TF32X3 = 3, MODE_TF32N_PACK = 4;
constexpr uint32_t SWZ_128B_BASE32B = 1;  // descriptor layout: 128-byte swizzle, 32-byte atoms

// PAIR: the TF32 form for a CTA pair (cta_group::2): one 256 x BN tile per pair, each CTA holding
// 128 rows of A and BN / 2 rows of B^T; the even CTA issues M = 256 MMAs that read both CTAs'
// shared memory and write 128 accumulator rows into each CTA's tensor memory.
template <int MODE, int BN, bool PAIR = false>
struct TfCfg {
    static constexpr bool TF = MODE != MODE_BF16X3;                  // a TF32 form
    static constexpr bool NMAJ = MODE == MODE_TF32N || MODE == MODE_TF32N_PACK;  // TF32 with B N-major
    static constexpr bool PACK = MODE == MODE_TF32N_PACK;
    static constexpr bool BN_MAJOR32 = NMAJ || MODE == MODE_TF32X3;  // B N-major, 32-bit
    static constexpr int BK = TF ? 32 : 64;                          // elements per 128-byte row
    static constexpr int TM = PAIR ? 2 * TF_BM : TF_BM;              // tile rows per work item
    static constexpr int B_ROWS = PAIR ? BN / 2 : BN;                // B rows held by one CTA
    static constexpr int A_BYTES = TF_BM * 128;                      // one A tile (16 KB)
    static constexpr int B_BYTES = B_ROWS * 128;                     // one B tile
    static constexpr int NOPS = (MODE == MODE_TF32 || NMAJ) ? 1 : 2;  // tiles per operand (hi, lo)
    static constexpr int STAGE_BYTES = NOPS * (A_BYTES + B_BYTES);
    static constexpr int STAGES = (4 * 49152) / STAGE_BYTES;         // 192 KB of operand stages
    // BN = 512 (TF32 N-major on CTA pairs): a 256 x 512 tile as two N = 256 MMAs per k step into
    // one 512-column accumulator -- 48 operand bytes per clock and SM at the full MMA rate instead
    // of 64, at the price of a single accumulator (the epilogue no longer overlaps the next tile)
    static_assert(BN <= 256 || (BN == 512 && PAIR && MODE == MODE_TF32N), "512-wide tiles: TF32N on CTA pairs");
    static constexpr int MMA_N = BN > 256 ? 256 : BN;                 // N of one MMA
    static constexpr int NACC = BN > 256 ? 1 : 2;                     // TMEM accumulators (512 columns)
    static constexpr int TMEM_COLS = NACC * BN;
    static constexpr int PACK_WARPS = 4;
    static constexpr int THREADS = PACK ? 192 + 32 * PACK_WARPS : 192;  // warps 6..: the packing warps
    static constexpr int STG_OFF = STAGES * STAGE_BYTES;      // epilogue staging: 4 warps x 2 x 4 KB
    static constexpr int STG_BYTES = 4 * 2 * 4096;
    static constexpr int BAR_OFF = STG_OFF + STG_BYTES;
    static constexpr int SMEM_BYTES = BAR_OFF + 512 + 1024;  // + barriers + alignment slack
    // instruction descriptor: D F32; TF32: A/B TF32, both K-major; BF16X3: A/B BF16, A K-major,
    // B MN-major; N = BN, M = 128
    static constexpr uint32_t IDESC =
        TF ? ((1u << 4) | (2u << 7) | (2u << 10) | (BN_MAJOR32 ? (1u << 16) : 0u) |
              ((uint32_t)(MMA_N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24))
            : ((1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(MMA_N >> 3) << 17) |
               ((uint32_t)(TM >> 4) << 24));
};

struct ItemPos {
    int leaf, tm, tn;
};

// Work item -> (leaf, tile row, tile column); tiles are TM rows high, taken in groups of
// TF_GROUP_M x 128 / TM tile rows (column-major inside a group) for L2 reuse of A and B.
template <int TM>
__device__ __forceinline__ ItemPos decode_item(const Leaf* __restrict__ leaves, int nleaves, int item) {
    int lo = 0, hi = nleaves - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&leaves[mid].tile_begin) <= item) lo = mid; else hi = mid - 1;
    }
    constexpr int GROUP = TF_GROUP_M * TF_BM / TM;
    const Leaf* L = &leaves[lo];
    int local = item - __ldg(&L->tile_begin);
    int tiles_m = (__ldg(&L->m) + TM - 1) / TM;
    int tiles_n = __ldg(&L->tiles_n);
    int per_group = GROUP * tiles_n;
    int g = local / per_group;
    int first_m = g * GROUP;
    int gsz = min(tiles_m - first_m, GROUP);
    int r = local - g * per_group;
    ItemPos p;
    p.leaf = lo;
    p.tm = first_m + r % gsz;
    p.tn = r / gsz;
    return p;
}

// Tile position of an item whose leaf is known (from an item -> leaf table: the resident mode's,
// or the one the planner writes for launches with many leaves); same order as decode_item.
template <int TM>
__device__ __forceinline__ ItemPos decode_in_leaf(const Leaf* __restrict__ leaves, int leaf, int item) {
    constexpr int GROUP = TF_GROUP_M * TF_BM / TM;
    const Leaf* L = &leaves[leaf];
    int local = item - __ldg(&L->tile_begin);
    int tiles_m = (__ldg(&L->m) + TM - 1) / TM;
    int tiles_n = __ldg(&L->tiles_n);
    int per_group = GROUP * tiles_n;
    int g = local / per_group;
    int first_m = g * GROUP;
    int gsz = min(tiles_m - first_m, GROUP);
    int r = local - g * per_group;
    ItemPos p;
    p.leaf = leaf;
    p.tm = first_m + r % gsz;
    p.tn = r / gsz;
    return p;
}

// Non-resident item: from the explicit layout (leaf and tile per item), the item -> leaf table, or
// a search over the leaves' tile ranges.
template <int TM>
__device__ __forceinline__ ItemPos decode_any(const Leaf* __restrict__ leaves, int nleaves, const ResidentCtl& ctl,
                                              int item) {
    if (ctl.item_tile) {
        const int t = __ldg(&ctl.item_tile[item]);
        ItemPos p;
        p.leaf = __ldg(&ctl.item_leaf[item]);
        p.tm = t >> 16;
        p.tn = t & 0xffff;
        return p;
    }
    if (ctl.item_leaf) return decode_in_leaf<TM>(leaves, __ldg(&ctl.item_leaf[item]), item);
    return decode_item<TM>(leaves, nleaves, item);
}

__device__ __forceinline__ unsigned ld_acquire_sys_u32(const volatile unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Resident mode: claim the next published item (compare-and-swap, so an exiting CTA never holds
// an unprocessed claim), or -1 on stop, error or `idle_ns` without new work.  `pub` caches the
// published count: it only grows while the kernel runs, so host memory is read only when the
// claims have caught up with the cached value.
__device__ __forceinline__ int res_claim(const ResidentCtl& c, unsigned& pub, int* err) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        const unsigned cur = *reinterpret_cast<volatile unsigned*>(c.next);
        if (cur >= pub) pub = ld_acquire_sys_u32(c.published);
        if (cur < pub) {
            if (atomicCAS(c.next, cur, cur + 1u) == cur) return (int)cur;
            continue;
        }
        if (*c.stop) return -1;
        if (error_raised(err)) return -1;
        if (globaltimer() - t0 > c.idle_ns) return -1;
        __nanosleep(1000);
    }
}

// Descriptors appended while the kernel runs: order the tensor-map reads after the claim.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
                 : "memory");
}

__device__ __forceinline__ const CUtensorMap* pick_map(const MapSet& maps, const CUtensorMap* gmaps, int idx) {
    return gmaps ? gmaps + idx : &maps.m[idx];
}

// Epilogue store of one 32 x 32 chunk (rows row_w.., columns col0..) into one target without a
// tensor map: the chunk sits row-major in shared memory (row stride 33 floats) and the warp writes
// it one row per step, lane j on column col0 + j, so every step is one contiguous 128-byte run.
__device__ __forceinline__ void store_chunk32(const Target& t, int row_w, int col0, const float* sf, int lane) {
    const int c = col0 + lane;
    if (c >= t.cols) return;
    const int nrow = min(32, t.rows - row_w);
    float* base = reinterpret_cast<float*>(t.c) + (long long)row_w * t.ldc + c;
    const float s = t.sign;
    for (int i = 0; i < nrow; ++i) {
        const float v = s * sf[i * 33 + lane];
        float* q = base + (long long)i * t.ldc;
        if (t.mode == TGT_STORE) *q = v;
        else if (t.mode == TGT_ATOMIC) atomicAdd(q, v);
        else *q += v;
    }
}

template <int MODE, int BN, bool RES, bool PAIR>
__global__ void __launch_bounds__(TfCfg<MODE, BN, PAIR>::THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ MapSet maps, const CUtensorMap* __restrict__ gmaps,
                     const Leaf* __restrict__ leaves, int nleaves, const Target* __restrict__ targets,
                     const CUtensorMap* __restrict__ tmaps, unsigned* __restrict__ flags,
                     int total_items, int* err, const ResidentCtl ctl) {
    static_assert(!PAIR || (MODE != MODE_TF32X3 && !RES), "CTA pairs: TF32 / split-BF16, non-resident only");
    using Cfg = TfCfg<MODE, BN, PAIR>;
    static_assert(!Cfg::PACK || (PAIR && !RES && BN == 256), "packing launches: 256 x 256 CTA-pair tiles");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t base_addr = (raw_addr + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_addr - raw_addr);
    // stage s: [A (hi) | A lo | B (hi) | B lo], 1024-byte aligned pieces
    auto stage_a = [&](int st, int op) { return base + st * Cfg::STAGE_BYTES + op * Cfg::A_BYTES; };
    auto stage_b = [&](int st, int op) {
        return base + st * Cfg::STAGE_BYTES + Cfg::NOPS * Cfg::A_BYTES + op * Cfg::B_BYTES;
    };
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + Cfg::BAR_OFF);
    uint64_t* full = bars;                       // [STAGES]
    uint64_t* empty = bars + Cfg::STAGES;        // [STAGES]
    uint64_t* tfull = bars + 2 * Cfg::STAGES;    // [2]
    uint64_t* tempty = tfull + 2;                // [2]
    uint64_t* done = tempty + 2;                 // [1]
    uint64_t* ring_full = done + 1;              // [4] resident mode: item ring, producer -> consumers
    uint64_t* ring_empty = ring_full + 4;        // [4] consumers (MMA + 4 epilogue warps) -> producer
    volatile int* ring = reinterpret_cast<volatile int*>(ring_empty + 4);  // [4]
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(ring_empty + 4) + 4;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // CTA pairs: work unit = cluster; rank 0 (the leader) issues the MMAs and owns the
    // operand-full and accumulator-free barriers, rank 1 holds the other half of each tile.
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0u;
    const int unit = PAIR ? (int)cluster_id_x() : (int)blockIdx.x;
    const int nunits = PAIR ? (int)nclusters_x() : (int)gridDim.x;
    // an explicit work layout holds only for the number of units it was planned for
    const bool layout_ok = RES || !ctl.item_tile || nunits == ctl.units;
    // ordering counters: flags[0] holds the epoch of the last completed launch, flags[1] counts the
    // CTAs that have finished this one, the per-tile counters follow; every launch (a graph replay
    // too) adds 4 to each counter it orders on, so this launch waits for 4 * (flags[0] + 1)
    unsigned* const ctr = flags ? flags + 2 : nullptr;
    const unsigned epoch = flags ? ld_acquire_u32(flags) + 1u : 0u;
    const int n_items = layout_ok ? total_items : 0;
    if (!layout_ok && threadIdx.x == 0) set_error(err, ERR_UNITS);

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], PAIR ? 8 : 4);  // epilogue warps (of both CTAs of a pair)
        }
        mbar_init(done, 1);
        for (int r = 0; r < 4; ++r) {
            mbar_init(&ring_full[r], 1);
            mbar_init(&ring_empty[r], 5);
        }
        fence_mbar_init();
    }
    if (warp == 1) {
        if (PAIR) {
            tmem_alloc_pair(tmem_holder, Cfg::TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_holder, Cfg::TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    if (PAIR) cluster_sync_all();  // the peer's barriers are initialised before any remote arrive
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(tmem_holder);

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            bool ok = true;
            int rslot = 0;
            uint32_t rph = 0;
            unsigned pub = 0;
            for (int item = RES ? -1 : unit;; item += RES ? 0 : nunits) {
                if (RES) {  // claim a published item and hand it to the consumers
                    item = res_claim(ctl, pub, err);
                    if (!mbar_wait(&ring_empty[rslot], rph ^ 1u, err, ERR_WAIT_EMPTY)) break;
                    ring[rslot] = item;
                    mbar_arrive(&ring_full[rslot]);
                    if (++rslot == 4) { rslot = 0; rph ^= 1u; }
                    if (item < 0) break;
                } else if (item >= n_items || !ok) {
                    break;
                }
                const ItemPos ip = RES ? decode_in_leaf<Cfg::TM>(leaves, __ldcg(&ctl.item_leaf[item]), item)
                                       : decode_any<Cfg::TM>(leaves, nleaves, ctl, item);
                const Leaf* L = &leaves[ip.leaf];
                const int am = __ldg(&L->a_map), bm = __ldg(&L->b_map);
                const int a_row = __ldg(&L->a_row) + ip.tm * Cfg::TM + (int)rank * TF_BM;
                const int a_col = __ldg(&L->a_col);
                // TF32: B^T, rows are N, columns K.  BF16X3 / TF32N: B as stored, rows K, columns N.
                const int b_row = __ldg(&L->b_row) + (MODE == MODE_TF32 ? ip.tn * BN + (int)rank * Cfg::B_ROWS : 0);
                // a pair's CTA holds half of every MMA's N columns: 128 of each 256 (BN = 512: B chunk
                // c of rank r is tile column (c / 4) * 256 + r * 128 + (c % 4) * 32)
                const int b_col = __ldg(&L->b_col) +
                                  (MODE == MODE_TF32 ? 0 : ip.tn * BN + (int)rank * (Cfg::B_ROWS < 128 ? Cfg::B_ROWS : 128));
                const int kb_n = __ldg(&L->kblocks);
                if (Cfg::PACK) {  // operands packed in this launch: their tiles are complete first
                    const int ja = __ldg(&L->a_job), jb = __ldg(&L->b_job);
                    if (ja >= 0) ok &= wait_counter(ctr + ja, epoch * (unsigned)ctl.pack_jobs[ja].pad_, err, ERR_ORDER);
                    if (jb >= 0) ok &= wait_counter(ctr + jb, epoch * (unsigned)ctl.pack_jobs[jb].pad_, err, ERR_ORDER);
                    fence_async_global();  // the packing warps' stores -> this CTA's TMA loads
                    if (!ok) break;
                }
                // TMA x coordinates must be 16-byte aligned (4 FP32 / 8 BF16 elements)
                if (((a_col | b_col) & (Cfg::TF ? 3 : 7)) != 0) {
                    set_error(err, ERR_ALIGN);
                    ok = false;
                    break;
                }
                if (RES) {
#pragma unroll
                    for (int op = 0; op < Cfg::NOPS; ++op) {
                        tensormap_acquire(pick_map(maps, gmaps, am * Cfg::NOPS + op));
                        tensormap_acquire(pick_map(maps, gmaps, bm * Cfg::NOPS + op));
                    }
                }
                for (int kb = 0; kb < kb_n; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, err, ERR_WAIT_EMPTY)) { ok = false; break; }
                    if (PAIR) {
                        // both halves land on the leader's full barrier
                        if (leader) mbar_arrive_expect_tx(&full[stage], 2 * Cfg::STAGE_BYTES);
                        const uint32_t fb = mapa_shared(smem_u32(&full[stage]), 0u);
                        if (MODE == MODE_BF16X3) {
#pragma unroll
                            for (int op = 0; op < 2; ++op) {  // hi, lo
                                const CUtensorMap* ma = pick_map(maps, gmaps, am * 2 + op);
                                const CUtensorMap* mb = pick_map(maps, gmaps, bm * 2 + op);
                                tma_load_2d_pair(stage_a(stage, op), ma, fb, a_col + kb * Cfg::BK, a_row);
#pragma unroll
                                for (int c = 0; c < Cfg::B_ROWS / 64; ++c)  // 64 N-columns x 64 K-rows per box
                                    tma_load_2d_pair(stage_b(stage, op) + c * 8192, mb, fb, b_col + c * 64,
                                                     b_row + kb * Cfg::BK);
                            }
                            ++issued;
                            if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1u; }
                            continue;
                        }
                        tma_load_2d_pair(stage_a(stage, 0), pick_map(maps, gmaps, am), fb, a_col + kb * Cfg::BK,
                                         a_row);
                        if (Cfg::NMAJ) {
#pragma unroll
                            for (int c = 0; c < Cfg::B_ROWS / 32; ++c)  // 32 N-columns x 32 K-rows per box
                                tma_load_2d_pair(stage_b(stage, 0) + c * 4096, pick_map(maps, gmaps, bm), fb,
                                                 b_col + (c >> 2) * 256 + (c & 3) * 32, b_row + kb * Cfg::BK);
                        } else {
                            tma_load_2d_pair(stage_b(stage, 0), pick_map(maps, gmaps, bm), fb, b_col + kb * Cfg::BK,
                                             b_row);
                        }
                        ++issued;
                        if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1u; }
                        continue;
                    }
                    mbar_arrive_expect_tx(&full[stage], Cfg::STAGE_BYTES);
#pragma unroll
                    for (int op = 0; op < Cfg::NOPS; ++op) {
                        const CUtensorMap* ma = pick_map(maps, gmaps, am * Cfg::NOPS + op);
                        const CUtensorMap* mb = pick_map(maps, gmaps, bm * Cfg::NOPS + op);
                        tma_load_2d(stage_a(stage, op), ma, &full[stage], a_col + kb * Cfg::BK, a_row);
                        if (MODE == MODE_TF32) {
                            tma_load_2d(stage_b(stage, op), mb, &full[stage], b_col + kb * Cfg::BK, b_row);
                        } else if (Cfg::BN_MAJOR32) {
#pragma unroll
                            for (int c = 0; c < BN / 32; ++c)  // 32 N-columns (128 B) x 32 K-rows per box
                                tma_load_2d(stage_b(stage, op) + c * 4096, mb, &full[stage], b_col + c * 32,
                                            b_row + kb * Cfg::BK);
                        } else {
#pragma unroll
                            for (int c = 0; c < BN / 64; ++c)  // 64 N-columns (128 B) x 64 K-rows per box
                                tma_load_2d(stage_b(stage, op) + c * 8192, mb, &full[stage], b_col + c * 64,
                                            b_row + kb * Cfg::BK);
                        }
                    }
                    ++issued;
                    if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
            }
            // drain: every issued copy must have landed before the CTA may exit (a pair: the
            // leader's MMAs have consumed it, which the stage's empty barrier reports in both CTAs)
            int s = stage;
            uint32_t ph = phase;
            for (int i = 0; i < min(issued, Cfg::STAGES); ++i) {
                if (--s < 0) { s = Cfg::STAGES - 1; ph ^= 1u; }
                mbar_wait(PAIR ? &empty[s] : &full[s], ph, err, ERR_WAIT_DRAIN);
            }
        }
    } else if (Cfg::PACK && warp >= 6) {
        // ------------------------------------------------------------ operand packing
        // Every packing warp of the launch takes chunks of PCH consecutive pack tiles, round robin
        // in job order (the launch's item order, so the tiles the first items wait for come first),
        // walking the jobs forward as its tile index grows.  A 64 x 64 tile in two passes of 32
        // rows x 64 columns (lane = column c0 + lane and c0 + lane + 32: 128-byte runs), all 64
        // loads of a pass before its stores.  After a chunk its stores are fenced for the async
        // proxy (TMA reads them) and lane 0 counts its tiles on their jobs' counters.
        constexpr int PCH = 8;
        const int gw = (int)blockIdx.x * Cfg::PACK_WARPS + (warp - 6), nw = (int)gridDim.x * Cfg::PACK_WARPS;
        int lo = 0;
        CopyJob J;
        J.tile_begin = -1;
        for (int t0 = gw * PCH; t0 < ctl.pack_tiles; t0 += nw * PCH) {
            const int t1 = min(t0 + PCH, ctl.pack_tiles);
            int first_job = -1, n_first = 0;  // the job whose tiles this chunk has done, and how many
#pragma unroll 1
            for (int t = t0; t < t1; ++t) {
                while (lo + 1 < ctl.pack_njobs && __ldg(&ctl.pack_jobs[lo + 1].tile_begin) <= t) {
                    ++lo;
                    if (first_job >= 0 && lo != first_job) {  // count what is done so far
                        fence_async_global();
                        __syncwarp();
                        if (lane == 0) {
                            __threadfence();
                            red_release_add_u32(ctr + first_job, (unsigned)n_first);
                        }
                        first_job = -1;
                        n_first = 0;
                    }
                }
                if (J.tile_begin != __ldg(&ctl.pack_jobs[lo].tile_begin)) J = ctl.pack_jobs[lo];  // increasing
                if (first_job < 0) first_job = lo;
                const int lt = t - J.tile_begin;
                const int tiles_c = (J.out_cols + 63) / 64;
                const int r0 = (lt / tiles_c) * 64, c0 = (lt % tiles_c) * 64 + lane;
                const float* x = static_cast<const float*>(J.x);
                float* out = static_cast<float*>(J.out);
#pragma unroll 1
                for (int half = 0; half < 2; ++half) {
                    const int rb = r0 + half * 32;
                    float v[2][32];
#pragma unroll
                    for (int p = 0; p < 32; ++p)
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int r = rb + p, c = c0 + 32 * u;
                            v[u][p] = (r < J.src_rows && c < J.src_cols) ? __ldcs(x + (long long)r * J.ldx + c) : 0.f;
                        }
#pragma unroll
                    for (int p = 0; p < 32; ++p)
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int r = rb + p, c = c0 + 32 * u;
                            if (r < J.out_rows && c < J.out_cols) out[(long long)r * J.ldo + c] = v[u][p];
                        }
                }
                ++n_first;
            }
            if (first_job >= 0) {
                fence_async_global();
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    red_release_add_u32(ctr + first_job, (unsigned)n_first);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            int rslot = 0;
            uint32_t rph = 0;
            for (int item = RES ? -1 : unit;; item += RES ? 0 : nunits, ++local) {
                if (RES) {
                    if (!mbar_wait(&ring_full[rslot], rph, err, ERR_WAIT_FULL)) break;
                    item = ring[rslot];
                    mbar_arrive(&ring_empty[rslot]);
                    if (++rslot == 4) { rslot = 0; rph ^= 1u; }
                    if (item < 0) break;
                } else if (item >= n_items || !ok) {
                    break;
                }
                const ItemPos ip = RES ? decode_in_leaf<Cfg::TM>(leaves, __ldcg(&ctl.item_leaf[item]), item)
                                       : decode_any<Cfg::TM>(leaves, nleaves, ctl, item);
                const int kb_n = __ldg(&leaves[ip.leaf].kblocks);
                const uint32_t cont = __ldg(&leaves[ip.leaf].cont) != 0 ? 1u : 0u;  // keep the chain's sum
                const int acc = local % Cfg::NACC;
                const uint32_t acc_phase = (local / Cfg::NACC) & 1;
                if (!mbar_wait(&tempty[acc], acc_phase ^ 1u, err, ERR_WAIT_ACC_FREE)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                for (int kb = 0; kb < kb_n; ++kb) {
                    if (!mbar_wait(&full[stage], phase, err, ERR_WAIT_FULL)) { ok = false; break; }
                    tc_fence_after();
                    if (MODE == MODE_TF32X3) {
                        const uint32_t ah = smem_u32(stage_a(stage, 0)), al = smem_u32(stage_a(stage, 1));
                        const uint32_t bh = smem_u32(stage_b(stage, 0)), bl = smem_u32(stage_b(stage, 1));
#pragma unroll
                        for (int kk = 0; kk < TF_BK / 8; ++kk) {  // K = 8 per MMA
                            const uint64_t dah = make_sdesc(ah + kk * 32, 16, 1024, SWZ_128B);
                            const uint64_t dal = make_sdesc(al + kk * 32, 16, 1024, SWZ_128B);
                            const uint64_t dbh = make_sdesc(bh + kk * 1024, 4096, 512, SWZ_128B_BASE32B);
                            const uint64_t dbl = make_sdesc(bl + kk * 1024, 4096, 512, SWZ_128B_BASE32B);
                            mma_tf32(d_tmem, dal, dbh, Cfg::IDESC, (kb | kk) != 0 ? 1u : 0u);  // lo * hi
                            mma_tf32(d_tmem, dah, dbl, Cfg::IDESC, 1u);                           // hi * lo
                            mma_tf32(d_tmem, dah, dbh, Cfg::IDESC, 1u);                           // hi * hi
                        }
                    } else if (Cfg::TF) {
                        const uint32_t a_addr = smem_u32(stage_a(stage, 0));
                        const uint32_t b_addr = smem_u32(stage_b(stage, 0));
#pragma unroll
                        for (int kk = 0; kk < TF_BK / 8; ++kk) {  // K = 8 per MMA, 32 bytes
                            const uint64_t ad = make_sdesc(a_addr + kk * 32, 16, 1024, SWZ_128B);
                            // TF32N: 8 K-rows of 128 bytes per step, read as two 4-row groups
                            // 512 bytes apart; 32-column chunks 4 KB apart
                            const uint64_t bd = Cfg::NMAJ
                                                    ? make_sdesc(b_addr + kk * 1024, 4096, 512, SWZ_128B_BASE32B)
                                                    : make_sdesc(b_addr + kk * 32, 16, 1024, SWZ_128B);
                            const uint32_t accum = ((kb | kk) != 0 ? 1u : 0u) | cont;
                            if (PAIR) {
                                mma_tf32_pair(d_tmem, ad, bd, Cfg::IDESC, accum);
                                if (BN > 256) {  // second N half: B chunks 4..7 (16 KB on), TMEM columns 256..511
                                    const uint64_t bd2 =
                                        make_sdesc(b_addr + kk * 1024 + 16384, 4096, 512, SWZ_128B_BASE32B);
                                    mma_tf32_pair(d_tmem + Cfg::MMA_N, ad, bd2, Cfg::IDESC, accum);
                                }
                            } else {
                                mma_tf32(d_tmem, ad, bd, Cfg::IDESC, accum);
                            }
                        }
                    } else {
                        const uint32_t ah = smem_u32(stage_a(stage, 0)), al = smem_u32(stage_a(stage, 1));
                        const uint32_t bh = smem_u32(stage_b(stage, 0)), bl = smem_u32(stage_b(stage, 1));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // K = 16 per MMA: 32 bytes of A, 16 rows of B
                            // A K-major: +32 B per step.  B N-major: 16 rows x 128 B per step,
                            // 64-column chunks 8 KB apart (LBO), 8-row groups 1 KB apart (SBO).
                            const uint64_t dah = make_sdesc(ah + kk * 32, 16, 1024, SWZ_128B);
                            const uint64_t dal = make_sdesc(al + kk * 32, 16, 1024, SWZ_128B);
                            const uint64_t dbh = make_sdesc(bh + kk * 2048, 8192, 1024, SWZ_128B);
                            const uint64_t dbl = make_sdesc(bl + kk * 2048, 8192, 1024, SWZ_128B);
                            const uint32_t first = ((kb | kk) != 0 ? 1u : 0u) | cont;
                            if (PAIR) {
                                mma_f16_pair(d_tmem, dal, dbh, Cfg::IDESC, first);  // lo * hi
                                mma_f16_pair(d_tmem, dah, dbl, Cfg::IDESC, 1u);     // hi * lo
                                mma_f16_pair(d_tmem, dah, dbh, Cfg::IDESC, 1u);     // hi * hi
                            } else {
                                mma_f16(d_tmem, dal, dbh, Cfg::IDESC, first);  // lo * hi
                                mma_f16(d_tmem, dah, dbl, Cfg::IDESC, 1u);     // hi * lo
                                mma_f16(d_tmem, dah, dbh, Cfg::IDESC, 1u);     // hi * hi
                            }
                        }
                    }
                    // stage is free once these MMAs have read it (in both CTAs of a pair)
                    if (PAIR) mma_commit_pair(&empty[stage], 3);
                    else mma_commit(&empty[stage]);
                    if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                // accumulator ready for the epilogue
                if (PAIR) mma_commit_pair(&tfull[acc], 3);
                else mma_commit(&tfull[acc]);
            }
            // drain: all MMAs issued by this thread must finish before TMEM is released (a pair
            // waits for this in both CTAs at the end)
            if (PAIR) {
                mma_commit_pair(done, 3);
            } else {
                mma_commit(done);
                mbar_wait(done, 0, err, ERR_WAIT_DRAIN);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..5)
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        uint8_t* stg = base + Cfg::STG_OFF + (warp - 2) * 8192;  // two 4 KB swizzled buffers
        int local = 0, chunk_ctr = 0;
        bool issued_bulk = false;
        bool last_mixed = false;  // the last TMA group read both staging buffers (a mixed-sign chunk)
        int rslot = 0;
        uint32_t rph = 0;
        for (int item = RES ? -1 : unit;; item += RES ? 0 : nunits, ++local) {
            if (RES) {
                int it = -1;
                if (lane == 0) {
                    if (mbar_wait(&ring_full[rslot], rph, err, ERR_WAIT_ACC)) it = ring[rslot];
                    mbar_arrive(&ring_empty[rslot]);
                }
                item = __shfl_sync(0xffffffffu, it, 0);
                if (++rslot == 4) { rslot = 0; rph ^= 1u; }
                if (item < 0) break;
            } else if (item >= n_items) {
                break;
            }
            const ItemPos ip = RES ? decode_in_leaf<Cfg::TM>(leaves, __ldcg(&ctl.item_leaf[item]), item)
                                   : decode_any<Cfg::TM>(leaves, nleaves, ctl, item);
            const Leaf* L = &leaves[ip.leaf];
            const int acc = local % Cfg::NACC;
            const uint32_t acc_phase = (local / Cfg::NACC) & 1;
            if (!mbar_wait(&tfull[acc], acc_phase, err, ERR_WAIT_ACC)) break;
            tc_fence_after();
            const int tb = __ldg(&L->tgt_begin), tc = __ldg(&L->tgt_count);
            bool has_pos = false, has_neg = false, all_tma = tmaps != nullptr;
            for (int t = 0; t < tc; ++t) {
                const float sg = __ldg(&targets[tb + t].sign);
                has_pos |= sg > 0.f;
                has_neg |= sg < 0.f;
                all_tma &= __ldg(&targets[tb + t].map) >= 0;
            }
            // this CTA's first row of the tile in its blocks (a pair: rank 1 holds rows 128..255)
            const int row_t = __ldg(&L->c_row0) + ip.tm * Cfg::TM + (int)rank * TF_BM;
            const int col_t = __ldg(&L->c_col0) + ip.tn * BN;      // the tile's first column
            const int row_w = row_t + q * 32;                        // this warp's first row
            const uint32_t t_base = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
            // contributions after a block's first write wait for that tile's write to complete
            bool ordered_ok = true, has_first = false;
            if (flags) {
                for (int t = 0; t < tc; ++t) {
                    const int fb = __ldg(&targets[tb + t].flag_base);
                    // no counter for a tile that lies outside a truncated block
                    if (fb < 0 || row_t >= __ldg(&targets[tb + t].rows) || col_t >= __ldg(&targets[tb + t].cols))
                        continue;
                    if (__ldg(&targets[tb + t].mode) == TGT_STORE) { has_first = true; continue; }
                    if (lane == 0) {
                        const int idx = fb + (row_t / TF_BM) * __ldg(&targets[tb + t].flag_cols) + col_t / BN;
                        ordered_ok &= wait_counter(ctr + idx, 4u * epoch, err, ERR_ORDER);
                    }
                }
                if (lane == 0) fence_async_global();
                ordered_ok = __shfl_sync(0xffffffffu, ordered_ok ? 1 : 0, 0) != 0;
            }
            // one 32-column chunk: staged and stored into every target
            auto emit_chunk = [&](int chunk, const uint32_t (&r)[32]) {
                const int col0 = col_t + chunk * 32;
                if (!ordered_ok) return;  // an expired wait: the device error word reports it
                if (all_tma) {
                    const bool mixed = has_pos && has_neg;
                    uint8_t* bpos;
                    uint8_t* bneg;
                    // a buffer is rewritten only once every TMA group that reads it has read it: with
                    // one buffer per chunk the group before last, after a mixed chunk (which reads
                    // both) all of them
                    if (mixed || last_mixed) {
                        if (lane == 0) bulk_wait_read<0>();
                    } else {
                        if (lane == 0) bulk_wait_read<1>();
                    }
                    if (mixed) {
                        bpos = stg;
                        bneg = stg + 4096;
                    } else {
                        bpos = bneg = stg + (chunk_ctr & 1) * 4096;
                    }
                    last_mixed = mixed;
                    __syncwarp();
                    // row `lane` of the chunk; 16-byte piece j sits at piece j ^ (row & 7)
                    const uint32_t row_off = (uint32_t)lane * 128u;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t off = row_off + ((uint32_t)(j ^ (lane & 7)) << 4);
                        const float4 v = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                                     __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                        if (has_pos) *reinterpret_cast<float4*>(bpos + off) = v;
                        if (has_neg && (mixed || !has_pos))
                            *reinterpret_cast<float4*>(bneg + off) = make_float4(-v.x, -v.y, -v.z, -v.w);
                    }
                    fence_async_shared();
                    __syncwarp();
                    if (lane == 0) {
                        for (int t = 0; t < tc; ++t) {
                            const Target& tg = targets[tb + t];
                            if (row_w >= tg.rows || col0 >= tg.cols) continue;
                            const CUtensorMap* m = tmaps + tg.map;
                            if (RES) tensormap_acquire(m);
                            const uint8_t* src = tg.sign > 0.f ? bpos : bneg;
                            if (tg.mode == TGT_STORE) tma_store_2d(m, src, col0, row_w);
                            else tma_reduce_add_2d(m, src, col0, row_w);
                        }
                        bulk_commit();
                        issued_bulk = true;
                    }
                    __syncwarp();
                    ++chunk_ctr;
                } else {
                    // no tensor map: stage the chunk row-major (lane = row), then coalesced rows
                    if (lane == 0 && issued_bulk) bulk_wait_read<0>();
                    __syncwarp();
                    float* sf = reinterpret_cast<float*>(stg);
#pragma unroll
                    for (int j = 0; j < 32; ++j) sf[lane * 33 + j] = __uint_as_float(r[j]);
                    __syncwarp();
                    for (int t = 0; t < tc; ++t) {
                        const Target tg = targets[tb + t];
                        if (row_w < tg.rows && col0 < tg.cols) store_chunk32(tg, row_w, col0, sf, lane);
                    }
                    __syncwarp();
                }
            };
            // TMEM loads double-buffered: chunk c + 1 is in flight while chunk c is stored
            constexpr int NCH = BN / 32;  // even
            uint32_t ra[32], rb[32];
            tmem_ld32(t_base, ra);
#pragma unroll 1
            for (int chunk = 0; chunk < NCH; chunk += 2) {
                tmem_ld_wait();
                tmem_ld32(t_base + (chunk + 1) * 32, rb);
                emit_chunk(chunk, ra);
                tmem_ld_wait();
                if (chunk + 2 < NCH) tmem_ld32(t_base + (chunk + 2) * 32, ra);
                emit_chunk(chunk + 1, rb);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR) mbar_arrive_cluster(mapa_shared(smem_u32(&tempty[acc]), 0u));
                else mbar_arrive(&tempty[acc]);
            }
            // first writes done: publish them tile by tile (one count per epilogue warp)
            if (flags && has_first) {
                if (lane == 0 && issued_bulk) bulk_wait<0>();  // this warp's TMA stores are complete
                fence_async_global();                           // ... and ordered before the count,
                __threadfence();                                // as are per-thread stores
                __syncwarp();
                if (lane == 0) {
                    for (int t = 0; t < tc; ++t) {
                        const int fb = __ldg(&targets[tb + t].flag_base);
                        if (fb < 0 || __ldg(&targets[tb + t].mode) != TGT_STORE) continue;
                        if (row_t >= __ldg(&targets[tb + t].rows) || col_t >= __ldg(&targets[tb + t].cols)) continue;
                        red_release_add_u32(ctr + fb + (row_t / TF_BM) * __ldg(&targets[tb + t].flag_cols) + col_t / BN,
                                            1u);
                    }
                }
                __syncwarp();
            }
            // resident mode: report the item once this warp's part of it is stored
            if (RES) {
                const int tag = __ldg(&L->tag);
                if (tag >= 0) {
                    if (lane == 0 && issued_bulk) bulk_wait<0>();
                    fence_async_global();
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) red_release_add_u32(ctl.done + tag, 1u);
                }
            }
            if (!ordered_ok) break;
        }
        // all bulk stores / reductions must be complete before the CTA (and its shared memory) ends
        if (lane == 0 && issued_bulk) bulk_wait<0>();
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    // the last CTA to finish publishes this launch's epoch for the next one (every CTA read the
    // old value at its start, before it finished)
    if (flags && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(flags + 1, 1u) == gridDim.x - 1) {
            flags[1] = 0u;
            __threadfence();
            red_release_add_u32(flags, 1u);
        }
    }
    if (PAIR) {
        // no MMA of the pair may still read this CTA's shared memory or write its tensor memory,
        // and neither CTA leaves while the other may still arrive on its barriers
        if (warp == 1 && lane == 0) mbar_wait(done, 0, err, ERR_WAIT_DRAIN);
        __syncwarp();
        tc_fence_before();
        cluster_sync_all();
        tc_fence_after();
        if (warp == 1) tmem_dealloc_pair(tmem_base, Cfg::TMEM_COLS);
        return;
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
    }
}

// One-time set-up of a kernel instance: its shared-memory size and, for CTA pairs, how many
// clusters of two fit on the GPU at once (one CTA per SM).
template <int MODE, int BN, bool RES, bool PAIR>
static cudaError_t tc_setup(int* pairs_out) {
    using Cfg = TfCfg<MODE, BN, PAIR>;
    auto kern = gemm_tc_kernel<MODE, BN, RES, PAIR>;
    static bool attr_set = false;
    static int max_pairs = 0;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if (PAIR) {
            // clusters of two that fit at once (one CTA per SM)
            cudaLaunchConfig_t q = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            q.gridDim = dim3(2 * 1024, 1, 1);
            q.blockDim = dim3(Cfg::THREADS, 1, 1);
            q.dynamicSmemBytes = Cfg::SMEM_BYTES;
            q.attrs = at;
            q.numAttrs = 1;
            e = cudaOccupancyMaxActiveClusters(&max_pairs, (void*)kern, &q);
            if (e != cudaSuccess) return e;
            if (max_pairs <= 0) return cudaErrorLaunchOutOfResources;
        }
        attr_set = true;
    }
    if (pairs_out) *pairs_out = max_pairs;
    return cudaSuccess;
}

template <int MODE, int BN, bool RES = false, bool PAIR = false>
static cudaError_t launch_tc_impl(const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                                  const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                                  int total_items, int* err, int grid, cudaStream_t stream,
                                  const ResidentCtl* ctl = nullptr, const int* item_leaf = nullptr,
                                  const int* item_tile = nullptr, int units = 0, const CopyJob* pack_jobs = nullptr,
                                  int pack_njobs = 0, int pack_tiles = 0) {
    using Cfg = TfCfg<MODE, BN, PAIR>;
    static_assert(Cfg::SMEM_BYTES <= 232448, "shared memory budget");
    auto kern = gemm_tc_kernel<MODE, BN, RES, PAIR>;
    int max_pairs = 0;
    cudaError_t se = tc_setup<MODE, BN, RES, PAIR>(&max_pairs);
    if (se != cudaSuccess) return se;
    ResidentCtl c;
    memset(&c, 0, sizeof(c));
    if (RES) {
        if (!ctl) return cudaErrorInvalidValue;
        c = *ctl;
    } else {
        if (total_items <= 0) return cudaSuccess;
        c.item_leaf = item_leaf;  // optional item -> leaf table (nullptr: binary search)
        c.item_tile = item_tile;  // optional explicit layout, planned for `units` units
        c.units = units;
        c.pack_jobs = pack_jobs;
        c.pack_njobs = pack_njobs;
        c.pack_tiles = pack_tiles;
        if (PAIR) grid = std::min(grid / 2, max_pairs);
        if (grid > total_items) grid = total_items;
        if (grid < 1) grid = 1;
        if (item_tile) grid = units;  // the layout's own unit count (the kernel checks it)
    }
    if (PAIR) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * grid, 1, 1);
        cfg.blockDim = dim3(Cfg::THREADS, 1, 1);
        cfg.dynamicSmemBytes = Cfg::SMEM_BYTES;
        cfg.stream = stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                           total_items, err, c);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    kern<<<grid, Cfg::THREADS, Cfg::SMEM_BYTES, stream>>>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                 total_items, err, c);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tf32_resident(const CUtensorMap* gmaps, const Leaf* leaves, const Target* targets,
                                      const CUtensorMap* tmaps, const ResidentCtl& ctl, int* err, int grid,
                                      cudaStream_t stream, bool nmajor) {
    MapSet none;
    memset(&none, 0, sizeof(none));
    if (nmajor)
        return launch_tc_impl<MODE_TF32N, 256, true>(none, gmaps, leaves, 0, targets, tmaps, nullptr, 0, err, grid,
                                                     stream, &ctl);
    return launch_tc_impl<MODE_TF32, 256, true>(none, gmaps, leaves, 0, targets, tmaps, nullptr, 0, err, grid,
                                                stream, &ctl);
}

cudaError_t launch_gemm_tf32(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                             const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                             int total_items, int* err, int grid, cudaStream_t stream, bool pair,
                             const int* item_leaf) {
    if (pair)
        return launch_tc_impl<MODE_TF32, 256, false, true>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                           total_items, err, grid, stream, nullptr, item_leaf);
    if (bn == 256)
        return launch_tc_impl<MODE_TF32, 256>(maps, gmaps, leaves, nleaves, targets, tmaps, flags, total_items,
                                              err, grid, stream, nullptr, item_leaf);
    return launch_tc_impl<MODE_TF32, 128>(maps, gmaps, leaves, nleaves, targets, tmaps, flags, total_items, err,
                                          grid, stream, nullptr, item_leaf);
}

cudaError_t launch_gemm_tf32n(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                              const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                              int total_items, int* err, int grid, cudaStream_t stream, bool pair,
                              const int* item_leaf, const int* item_tile, int units) {
    if (pair && bn == 512)
        return launch_tc_impl<MODE_TF32N, 512, false, true>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                            total_items, err, grid, stream, nullptr, item_leaf,
                                                            item_tile, units);
    if (pair)
        return launch_tc_impl<MODE_TF32N, 256, false, true>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                            total_items, err, grid, stream, nullptr, item_leaf,
                                                            item_tile, units);
    if (bn == 512) return cudaErrorInvalidValue;  // 512-wide tiles exist on CTA pairs only
    if (bn == 256)
        return launch_tc_impl<MODE_TF32N, 256>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                               total_items, err, grid, stream, nullptr, item_leaf, item_tile, units);
    return launch_tc_impl<MODE_TF32N, 128>(maps, gmaps, leaves, nleaves, targets, tmaps, flags, total_items,
                                           err, grid, stream, nullptr, item_leaf, item_tile, units);
}

cudaError_t launch_gemm_tf32n_pack(const CUtensorMap* gmaps, const Leaf* leaves, int nleaves, const Target* targets,
                                   const CUtensorMap* tmaps, unsigned* flags, int total_items, int* err, int grid,
                                   cudaStream_t stream, const int* item_leaf, const CopyJob* jobs, int njobs,
                                   int pack_tiles) {
    if (!flags || !jobs || njobs <= 0) return cudaErrorInvalidValue;  // the jobs' counters live in flags
    MapSet none;
    memset(&none, 0, sizeof(none));
    return launch_tc_impl<MODE_TF32N_PACK, 256, false, true>(none, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                             total_items, err, grid, stream, nullptr, item_leaf,
                                                             nullptr, 0, jobs, njobs, pack_tiles);
}

int gemm_tf32n_pair_units(int sms, int bn) {
    int max_pairs = 0;
    const cudaError_t e = bn == 512 ? tc_setup<MODE_TF32N, 512, false, true>(&max_pairs)
                                    : tc_setup<MODE_TF32N, 256, false, true>(&max_pairs);
    if (e != cudaSuccess || max_pairs <= 0) return 0;
    return std::min(sms / 2, max_pairs);
}

int gemm_bf16x3_pair_units(int sms) {
    int max_pairs = 0;
    if (tc_setup<MODE_BF16X3, 256, false, true>(&max_pairs) != cudaSuccess || max_pairs <= 0) return 0;
    return std::min(sms / 2, max_pairs);
}

cudaError_t launch_gemm_tf32x3(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                               const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                               int total_items, int* err, int grid, cudaStream_t stream, const int* item_leaf) {
    if (bn == 256)
        return launch_tc_impl<MODE_TF32X3, 256>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                total_items, err, grid, stream, nullptr, item_leaf);
    return launch_tc_impl<MODE_TF32X3, 128>(maps, gmaps, leaves, nleaves, targets, tmaps, flags, total_items,
                                            err, grid, stream, nullptr, item_leaf);
}

cudaError_t launch_gemm_bf16x3(int bn, const MapSet& maps, const CUtensorMap* gmaps, const Leaf* leaves, int nleaves,
                               const Target* targets, const CUtensorMap* tmaps, unsigned* flags,
                               int total_items, int* err, int grid, cudaStream_t stream, const int* item_leaf,
                               const int* item_tile, int units, bool pair) {
    if (pair)
        return launch_tc_impl<MODE_BF16X3, 256, false, true>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                             total_items, err, grid, stream, nullptr, item_leaf,
                                                             item_tile, units);
    if (bn == 256)
        return launch_tc_impl<MODE_BF16X3, 256>(maps, gmaps, leaves, nleaves, targets, tmaps, flags,
                                                total_items, err, grid, stream, nullptr, item_leaf, item_tile, units);
    return launch_tc_impl<MODE_BF16X3, 128>(maps, gmaps, leaves, nleaves, targets, tmaps, flags, total_items,
                                            err, grid, stream, nullptr, item_leaf, item_tile, units);
}

cudaError_t preload_gemm_tf32() {
    cudaError_t e = tc_setup<MODE_TF32, 128, false, false>(nullptr);
    return e != cudaSuccess ? e : tc_setup<MODE_TF32, 256, false, false>(nullptr);
}

int tf32_tile_m() { return TF_BM; }
int tf32_tile_k() { return TF_BK; }
int bf16x3_tile_k() { return 64; }

}  // namespace swk
