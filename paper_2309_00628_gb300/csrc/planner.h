// planner.h -- the planner that lowers one product (or a batch) to an op list: the materialised
// schedules (planner.cu) and the FUSED schedule with its accumulation chains and the batched
// grouped launch (fused.cu).
#pragma once

#include "host.h"

namespace swh {

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
    // Products of the top recursion level that take part (bit i: product i + 1 of Sec. 2.2 / 2.3,
    // Knuth's form in the BDPZ numbering); the others are left out and C holds the contributions of
    // the rest (FUSED only).  0x7F: the whole product.
    uint32_t top_mask = 0x7Fu;
    // B-side operand sums shared by products with the same B (the row panels of one product; FUSED,
    // TF32 leaves): 0 computed by the product itself; 1 only the B-side sums, written to b_sums (no
    // product); 2 read from b_sums (no B-side pass).
    int b_sums_mode = 0;
    char* b_sums = nullptr;

    // Batch mode: products append their leaves, targets and operand maps to one grouped launch
    // instead of emitting their own (operand maps then live in global memory).
    bool batch = false;
    bool server = false;  // plan for the serving loop (no ordering counters)
    int force_bn = 0;
    int sms = 0;              // SMs of the device (explicit work layouts are planned for its units)
    int batch_bn = 256;       // batched launch: tile width of the grouped GEMM (128 or 256)
    bool batch_pair = false;  // batched launch: CTA-pair form (256 x 256 tiles; N-major B only)
    // batched launch in the CTA-pair form, no recursion: the GEMM launch runs the packing copies
    // itself (each leaf's loads wait for its operands' pack jobs) instead of a copy launch before it
    bool pack_in_gemm = false;
    // The CTA-pair GEMM (cta_group::2; TF32 and split-BF16 leaves) serves single products with
    // 256-wide tiles; batched and serving launches keep the one-CTA form unless told otherwise.
    // SWMM_NO_PAIR=1 disables it (diagnostics).
    bool pair_ok(int bn) const {
        static const bool off = getenv("SWMM_NO_PAIR") != nullptr;
        return !off && (bn == 256 || (bn == 512 && nmaj && !bf)) && !batch && !server && !x3 && eb == 4;
    }
    // Tile width of a TF32 launch over C blocks `cols` wide: 512 (CTA pairs, one accumulator, a
    // quarter fewer operand bytes per MMA) where the blocks are at least 512 wide and 512-wide tiles
    // pad no more than 256-wide ones; else 256, or 128 for narrow blocks.  `shallow`: the leaves'
    // inner dimension is at most 2048 and each tile feeds several C blocks (recursive leaves), so
    // the one accumulator of a 512-wide tile would expose an epilogue as long as a good part of
    // the tile's MMA work: 256-wide tiles with two accumulators instead (n = 8192: Winograd L2
    // 1.770 -> 1.728 ms, L3 3.985 -> 3.760, Strassen L2 1.637 -> 1.573; with 4096-deep leaves
    // 512-wide tiles stay ahead, n = 16384 L2 10.41 vs 10.96 ms).
    int tf32_bn(int cols, bool shallow = false) const {
        if (bn_override()) return bn_override() == 512 && !pair_ok(512) ? 256 : bn_override();
        if (cols <= 128) return 128;
        if (!shallow && pair_ok(512) && cols >= 512 && round_up(cols, 512) == round_up(cols, 256)) return 512;
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

    // two independent block additions (z1 = x1 + s1 y1, z2 = x2 + s2 y2) in one launch; with
    // halves (FP32, split-BF16 leaves next) each z's bf16 hi / lo halves are written as well
    void add2(View z1, View x1, View y1, float s1, View z2, View x2, View y2, float s2,
              const View* h1 = nullptr, const View* l1 = nullptr, const View* h2 = nullptr,
              const View* l2 = nullptr) {
        Op o;
        o.kind = OP_ADDSUB2;
        o.eb = eb;
        o.job_a = {z1.rows, z1.cols, z1.p, z1.ld, x1.p, x1.ld, y1.p, y1.ld, s1};
        o.job_b = {z2.rows, z2.cols, z2.p, z2.ld, x2.p, x2.ld, y2.p, y2.ld, s2};
        if (h1) { o.job_a.zh = h1->p; o.job_a.zl = l1->p; o.job_a.ldh = h1->ld; }
        if (h2) { o.job_b.zh = h2->p; o.job_b.zl = l2->p; o.job_b.ldh = h2->ld; }
        push(o);
    }
    // z = x + s y and z's bf16 halves in one pass (one job of the two-job launch)
    void add_split(View z, View x, View y, float s, const View& hi, const View& lo) {
        Op o;
        o.kind = OP_ADDSUB2;
        o.eb = eb;
        o.job_a = {z.rows, z.cols, z.p, z.ld, x.p, x.ld, y.p, y.ld, s};
        o.job_a.zh = hi.p;
        o.job_a.zl = lo.p;
        o.job_a.ldh = hi.ld;
        o.job_b = {0, 0, nullptr, 0, nullptr, 0, nullptr, 0, 0.f};
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

    // ---------------------------------------------------------- leaves and materialised schedules (planner.cu)
    // A destination of a leaf product: block c receives sign * P (mode TGT_STORE: the block's first
    // write; TGT_ADD / TGT_ATOMIC: added; -1: decided by `written`).  All destinations of one leaf
    // have the product's shape.
    struct Dest { View c; float sign; int mode; };
    // leaf blocks of C already written by the plan (its launches run in order on one stream)
    std::set<std::tuple<const char*, int, int>> written;
    // One leaf product c (=|+=) a b: tensor cores (FP32), split leaves, or the SIMT kernel (FP64).
    bool gemm(View a, View b, View c, int mode);
    bool gemm_split(View a, View b, View c, int mode);
    bool simt(View a, View b, View c, int mode);
    // The same with several destinations (mode -1 resolved against `written`).
    bool leaf_to(View a, View b, std::vector<Dest> d);
    bool gemm_to(View a, View b, const std::vector<Dest>& d);
    bool gemm_split_to(View a, View b, const std::vector<Dest>& d);
    // the split leaf on halves made already (a, b: the FP32 operands' extents)
    bool gemm_split_halves(View a, View ah, View al, View bh, View bl, const std::vector<Dest>& d);
    // a block's first write stores, later ones add (the plan's launches run in order)
    void resolve_modes(std::vector<Dest>& d) {
        for (Dest& x : d)
            if (x.mode < 0)
                x.mode = written.insert(std::make_tuple(x.c.p, x.c.rows, x.c.cols)).second ? TGT_STORE : TGT_ADD;
    }
    bool simt_to(View a, View b, const std::vector<Dest>& d);
    // Table 2 with its post-additions (steps 13-17, 20, 22) folded into the epilogues of the
    // products: each product adds +-P into the C blocks it feeds (used for the level just above
    // the leaves; SWMM_TWO_TEMP_LITERAL=1: the table's steps one by one, for comparison).
    bool two_temp_folded(View a, View b, const std::vector<Dest>& d, int L);
    // c <- a b at depth L with the plan's schedule: Alg. 2 / Alg. 3 with fresh temporaries, Table 2
    // (two temporaries per level) or Table 3 (temporaries in A, B and C).
    bool product(View a, View b, View c, int L);
    bool alloc_strassen(View a, View b, View c, int L);
    bool alloc_winograd(View a, View b, View c, int L);
    bool two_temp(View a, View b, View c, int L);
    bool in_place(View a, View b, View c, int L);

    // ---------------------------------------------------------- FUSED (fused.cu)
    // Per-level coefficient tables of the 7 products.
    struct Term { int q; int s; };  // quadrant (0:11 1:12 2:21 3:22), sign
    struct ProdTab {
        int pure_a_q[7];  // quadrant of A if the A operand is a single block, else -1
        int pure_b_q[7];
        int ntgt[7];
        Term tgt[7][4];
    };
    static const ProdTab& table(int algo);
    // depth-1 accumulation chains (TF32 on CTA pairs, split-BF16); *done = 0: not applicable
    bool chain_plan(const ProdTab& T, Op o, View C, const std::vector<Leaf>& base, int mb, int nb, int bn,
                    const std::vector<int>& flag_base, const std::vector<int>& flag_cols, int nflags, int* done);
    // FUSED at depth 1..3: one operand-sum pass, one grouped launch over the 7^L leaves
    bool fused(View A, View B, View C, int L);
    // many products in one grouped launch
    bool batched(const sw_problem* probs, int count, const std::vector<int>& depth);
};

}  // namespace swh
