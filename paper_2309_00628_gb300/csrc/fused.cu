// fused.cu -- the FUSED schedule of the planner: the product tables of one level (Sec. 2.2, 2.3),
// all levels' operand sums in one pass, the 7^L leaf products in one grouped launch whose epilogue
// adds +-P into the C blocks (the post-additions), the depth-1 accumulation chains, and the batched
// grouped launch of many products.
#include "planner.h"

namespace swh {


const Planner::ProdTab& Planner::table(int algo) {
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
bool Planner::chain_plan(const ProdTab& T, Op o, View C, const std::vector<Leaf>& base, int mb, int nb, int bn,
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
bool Planner::fused(View A, View B, View C, int L) {
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
    auto in_mask = [&](int w) { return ((top_mask >> (w / (nleaf / 7))) & 1u) != 0; };
    for (int w = 0; w < nleaf; ++w) {
        if (!in_mask(w)) continue;  // a left-out top-level product: no operand slots, no leaf
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
    const bool share_b = b_sums_mode != 0 && eb == 4 && !bf && !x3 && !bt;
    View SB = split_sums ? View{nullptr, nb, nbs * kb, nb}
              : share_b  ? View{b_sums, nb, nbs * kb, nb}
              : bt       ? talloc(std::max(nbs, 1) * nb, kb)
                         : talloc(std::max(nbs, 1) * kb, nb);
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
    } else if (share_b && b_sums_mode == 1) {  // only the shared B-side sums
        if (nbs > 0) push(pb);
        return true;
    } else if (share_b) {                       // B-side sums already in b_sums
        if (na > 0) push(pa);
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
    const int bn_o = eb == 8                ? F64_BN
                     : force_bn             ? force_bn
                     : x3 || (bf && nb <= 128) ? 128
                     : bf                   ? 256
                                            : tf32_bn(nb, kb <= 2048);
    // Ordered stores pay off only while every unit starts on a first writer's work: a product with
    // fewer first-writer jobs than units leaves the other units waiting for those stores (n = 4096,
    // depth 1: 32 store jobs for 76 CTA pairs), so it zeroes C and reduce-adds everything instead.
    bool ordered = eb == 4 && L == 1 && !batch && !server && top_mask == 0x7Fu;
    if (ordered) {
        const bool pr = !bf && !x3 && pair_ok(bn_o);
        const long long tm_rows = pr ? 2LL * tf32_tile_m() : tf32_tile_m();
        const long long positions = ceil_div(mb, tm_rows) * ceil_div(nb, bn_o);
        const long long store_jobs = ceil_div(positions, bn_o > 256 ? 1 : 2);
        const int units = pr ? gemm_tf32n_pair_units(sms, bn_o) : sms;
        if (units > 0 && store_jobs < units) ordered = false;
    }
    if (!ordered) memset0(C);
    std::vector<int> first_writer(1 << (2 * L), -1), flag_base(1 << (2 * L), -1), flag_cols(1 << (2 * L), 0);
    int nflags = 0;
    // leaves and their Kronecker-product targets
    std::vector<Leaf> base_leaves;
    std::vector<Target> tg;
    const int tm_sz = eb == 4 ? tf32_tile_m() : F64_BM;
    const int bn = bn_o;
    for (int w = 0; w < nleaf; ++w) {
        if (!in_mask(w)) continue;
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
// all products go into a single persistent GEMM launch (longest k first).  With pack_in_gemm (no
// recursion, CTA pairs) that launch runs the packing copies itself, in product order, and each
// leaf's loads wait for its operands' jobs.  C needs no staging: unaligned or ragged C blocks take
// the per-thread epilogue.
bool Planner::batched(const sw_problem* probs, int count, const std::vector<int>& depth) {
    batch = true;
    force_bn = batch_bn == 128 ? 128 : 256;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].k > probs[y].k; });
    std::vector<CopyJob> packs, trans;
    int pack_tiles = 0, trans_tiles = 0;
    std::vector<View> As(count), Bs(count), Cs(count);
    std::vector<int> ajob(count, -1), bjob(count, -1);  // pack job of each product's A / B
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
            ajob[i] = (int)packs.size();
            packs.push_back(job(a, a2, pack_tiles));
            a = a2;
        }
        if (nmaj) {  // B read as stored: packed only when its rows are not 16-byte aligned
            if (!vec_ok(b)) {
                View b2 = talloc(q.k, q.n);
                bjob[i] = (int)packs.size();
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
    bool depth0 = true;
    for (int i = 0; i < count; ++i) depth0 &= depth[i] == 0;
    const bool in_gemm = pack_in_gemm && batch_pair && nmaj && depth0 && !packs.empty();
    for (size_t j = 0; j < packs.size(); ++j)  // tile counts, for the in-launch form's counters
        packs[j].pad_ = (j + 1 < packs.size() ? packs[j + 1].tile_begin : pack_tiles) - packs[j].tile_begin;
    if (!dry) {
        for (int t = in_gemm ? 1 : 0; t < 2; ++t) {
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
        const size_t nl = bleaves.size();
        const bool ok = depth[i] == 0 ? gemm(As[i], Bs[i], c, TGT_STORE) : fused(As[i], Bs[i], c, depth[i]);
        if (!ok) return false;
        for (size_t l = nl; l < bleaves.size(); ++l) {
            bleaves[l].a_job = in_gemm ? ajob[i] : -1;
            bleaves[l].b_job = in_gemm ? bjob[i] : -1;
        }
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
    if (in_gemm) {
        o.pack = true;
        o.njobs = (int)packs.size();
        o.tiles = pack_tiles;
        o.jobs_off = put_blob(packs.data(), packs.size() * sizeof(CopyJob));
    }
    batch = false;  // the combined op itself is emitted normally
    emit_grouped(o, bleaves, btargets, in_gemm ? (int)packs.size() : 0);  // in_gemm: one counter per job
    return true;
}

// Elements of the B-side operand sums of a FUSED FP32 product with TF32 leaves at depth L (the
// slot stack fused() writes: one (k/2^L rounded to the k-block) x (n/2^L rounded to 4) slot per
// leaf whose B operand is a sum).
long long fused_b_sum_elems(int algo, int k, int n, int L) {
    const Planner::ProdTab& T = Planner::table(algo);
    const long long s = 1LL << L;
    const long long kb = round_up(ceil_div(k, s), tf32_tile_k()), nb = round_up(ceil_div(n, s), 4);
    int nleaf = 1;
    for (int i = 0; i < L; ++i) nleaf *= 7;
    long long nbs = 0;
    for (int w = 0; w < nleaf; ++w) {
        bool pure = true;
        for (int l = 0, div = nleaf / 7; l < L; ++l, div /= 7)
            if (T.pure_b_q[(w / div) % 7] < 0) pure = false;
        if (!pure) ++nbs;
    }
    return nbs * kb * nb;
}

}  // namespace swh
