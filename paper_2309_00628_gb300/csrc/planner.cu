// planner.cu -- tensor-map encoding, the leaf launches and the materialised schedules of the
// planner (Alg. 2 / Alg. 3 allocating, Table 2, Table 3), the recursion depth (Sec. 3.4 cutoff) and
// the construction of a product's plan (odd sizes: Sec. 3.1 padding, or peeling).
#include "planner.h"

namespace swh {

// ------------------------------------------------------------------ tensor-map encoding
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

// One leaf product c (=|+=) a b on the tensor cores (FP32: b as stored, or as B^T in bt
// storage) or, for FP64, on the SIMT kernel.
bool Planner::gemm(View a, View b, View c, int mode) { return leaf_to(a, b, {Dest{c, 1.f, mode}}); }
bool Planner::gemm_split(View a, View b, View c, int mode) { return gemm_split_to(a, b, {Dest{c, 1.f, mode}}); }
bool Planner::simt(View a, View b, View c, int mode) { return simt_to(a, b, {Dest{c, 1.f, mode}}); }

bool Planner::leaf_to(View a, View b, std::vector<Dest> d) {
    resolve_modes(d);
    if (eb == 8) return simt_to(a, b, d);
    if (bf || x3) return gemm_split_to(a, b, d);
    return gemm_to(a, b, d);
}

// TF32 leaf on the tensor cores, one launch, the product added into every destination.
bool Planner::gemm_to(View a, View b, const std::vector<Dest>& d) {
    const int rows = d[0].c.rows, cols = d[0].c.cols;
    if (rows <= 0 || cols <= 0) return true;
    if (a.cols == 0) {
        for (const Dest& x : d)
            if (x.mode == TGT_STORE) memset0(x.c);
        return true;
    }
    if (dry) return true;
    std::vector<Target> tv;
    for (const Dest& x : d) tv.push_back(make_target(x.c, x.sign, x.mode, target_map(x.c)));
    Leaf lf;
    memset(&lf, 0, sizeof(lf));
    lf.tag = -1;
    lf.a_map = 0;
    lf.b_map = 1;
    lf.m = rows;
    lf.n = cols;
    lf.tgt_begin = 0;
    lf.tgt_count = (int)tv.size();
    lf.tile_begin = 0;
    Op o;
    o.kind = OP_GEMM_TF32;
    o.bn = force_bn ? force_bn : tf32_bn(cols, d.size() > 1 && a.cols <= 2048);
    lf.kblocks = (int)ceil_div(a.cols, tf32_tile_k());
    lf.tiles_n = (int)ceil_div(cols, o.bn);
    o.nmaj = nmaj;
    if (!make_map_f32(&o.maps.m[0], a.p, a.rows, a.cols, a.ld, 32, tf32_tile_m()) ||
        !(nmaj ? make_map_f32_n(&o.maps.m[1], b.p, b.rows, b.cols, b.ld)
               : make_map_f32(&o.maps.m[1], b.p, b.rows, b.cols, b.ld, 32, b_box(o.bn)))) {
        err = "tensor map encoding failed (alignment?)";
        return false;
    }
    o.items = (int)(ceil_div(rows, tf32_tile_m()) * lf.tiles_n);
    std::vector<Leaf> lv(1, lf);
    if (pair_ok(o.bn)) to_pair(o, lv);
    emit_grouped(o, lv, tv, 0);
    return true;
}

// Split leaf (split-BF16 or compensated TF32): both operands split into (hi, lo) halves in
// workspace (released once the launch is queued: later ops run after it on the same stream),
// then one launch.
bool Planner::gemm_split_to(View a, View b, const std::vector<Dest>& d) {
    const int rows = d[0].c.rows, cols = d[0].c.cols;
    if (rows <= 0 || cols <= 0) return true;
    if (a.cols == 0) {
        for (const Dest& x : d)
            if (x.mode == TGT_STORE) memset0(x.c);
        return true;
    }
    const size_t mark = ws_top;
    View ah, al, bh, bl;
    split(a, ah, al);
    split(b, bh, bl);
    const bool ok = gemm_split_halves(a, ah, al, bh, bl, d);
    ws_top = mark;
    return ok;
}

bool Planner::gemm_split_halves(View a, View ah, View al, View bh, View bl, const std::vector<Dest>& d) {
    const int rows = d[0].c.rows, cols = d[0].c.cols;
    if (rows <= 0 || cols <= 0) return true;
    bool ok = true;
    if (!dry) {
        std::vector<Target> tv;
        for (const Dest& x : d) tv.push_back(make_target(x.c, x.sign, x.mode, target_map(x.c)));
        Leaf lf;
        memset(&lf, 0, sizeof(lf));
        lf.tag = -1;
        lf.a_map = 0;
        lf.b_map = 1;
        lf.m = rows;
        lf.n = cols;
        lf.tgt_count = (int)tv.size();
        Op o;
        o.kind = x3 ? OP_GEMM_TF32X3 : OP_GEMM_BF16X3;
        o.bn = bn_override() ? bn_override() : (x3 || cols <= 128 ? 128 : 256);
        lf.kblocks = (int)ceil_div(a.cols, x3 ? tf32_tile_k() : bf16x3_tile_k());
        lf.tiles_n = (int)ceil_div(cols, o.bn);
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
        o.items = (int)(ceil_div(rows, tf32_tile_m()) * lf.tiles_n);
        if (!x3 && pair_ok(o.bn)) {  // 256-row tiles on CTA pairs
            o.items = (int)(ceil_div(rows, 2 * tf32_tile_m()) * lf.tiles_n);
            o.pair = true;
        }
        o.nleaves = 1;
        o.leaves_off = put_blob(&lf, sizeof(lf));
        o.targets_off = put_blob(tv.data(), tv.size() * sizeof(Target));
        flush_tmaps(o);
        push(o);
    }
    return ok;
}

// SIMT product (FP64 leaves; FP32 thin fix-ups) with b in logical orientation (k x n).
bool Planner::simt_to(View a, View b, const std::vector<Dest>& d) {
    const int rows = d[0].c.rows, cols = d[0].c.cols;
    if (rows <= 0 || cols <= 0) return true;
    if (a.cols == 0) {
        for (const Dest& x : d)
            if (x.mode == TGT_STORE) memset0(x.c);
        return true;
    }
    if (dry) return true;
    std::vector<Target> tv;
    for (const Dest& x : d) tv.push_back(make_target(x.c, x.sign, x.mode));
    Leaf lf;
    memset(&lf, 0, sizeof(lf));
    lf.tag = -1;
    lf.a_map = 0;
    lf.b_map = 1;
    lf.m = rows;
    lf.n = cols;
    lf.kblocks = a.cols;
    lf.tiles_n = (int)ceil_div(cols, F64_BN);
    lf.tgt_count = (int)tv.size();
    Op o;
    o.kind = OP_GEMM_SIMT;
    o.eb = eb;
    o.wtile = wtile && eb == 8;
    MatRef refs[2] = {{a.p, a.ld, a.rows, a.cols}, {b.p, b.ld, b.rows, b.cols}};
    o.refs_off = put_blob(refs, sizeof(refs));
    o.items = (int)(ceil_div(rows, F64_BM) * lf.tiles_n);
    o.nleaves = 1;
    o.leaves_off = put_blob(&lf, sizeof(lf));
    o.targets_off = put_blob(tv.data(), tv.size() * sizeof(Target));
    push(o);
    return true;
}

// ---------------------------------------------------------- materialised schedules
bool Planner::product(View a, View b, View c, int L) {
    if (L == 0) return gemm(a, b, c, TGT_STORE);
    if (fused_below > 0 && L <= fused_below) {
        // the fused bottom of a deep FUSED product; its sum slots are free again once its
        // launches are queued (everything after it runs later on the same stream)
        const size_t mark = ws_top;
        const bool ok = fused(a, b, c, L);
        ws_top = mark;
        return ok;
    }
    if (fused_below > 0 && algo == SW_ALGO_WINOGRAD) return two_temp(a, b, c, L);
    if (sched == SW_SCHED_TWO_TEMP) {
        // Table 2 step by step down to one level above the leaves; that last level folds its
        // post-additions into the leaf epilogues (deeper folding multiplies the C blocks every leaf
        // launch writes: measured slower at depth 2).  The product overwrites c, so none of its
        // blocks counts as written yet.
        static const bool literal = getenv("SWMM_TWO_TEMP_LITERAL") != nullptr;  // diagnostics
        if (literal || L > 1) return two_temp(a, b, c, L);
        written.clear();
        return two_temp_folded(a, b, {Dest{c, 1.f, -1}}, L);
    }
    if (sched == SW_SCHED_IN_PLACE) return in_place(a, b, c, L);
    return algo == SW_ALGO_STRASSEN ? alloc_strassen(a, b, c, L) : alloc_winograd(a, b, c, L);
}

// Alg. 2 (Sec. 2.2) with fresh temporaries: two operand sums, seven products.
bool Planner::alloc_strassen(View a, View b, View c, int L) {
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
bool Planner::alloc_winograd(View a, View b, View c, int L) {
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
bool Planner::two_temp(View a, View b, View c, int L) {
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

// Table 2 (Sec. 3.3) with the post-additions folded into the products' epilogues.  The sums take
// the table's steps and order on X (A-quadrant sums) and Y (B-quadrant sums), two sum steps per
// launch where the table has two in a row; each product adds sign * P straight into the C blocks
// its U-chain terms reach (BDPZ coefficients, Sec. 2.3), the block's first write storing, so steps
// 13-17, 20 and 22 need no launch of their own and P1 no longer occupies X.  `d` is where this
// product goes: the quadrant destinations of the level above, its sign folded in (at the top, C
// itself).  Footprint per level: X (m/2 x k/2) and Y (k/2 x n/2).
bool Planner::two_temp_folded(View a, View b, const std::vector<Dest>& d, int L) {
    if (L == 0) return leaf_to(a, b, d);
    View A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
    View B11 = quadB(b, 0), B12 = quadB(b, 1), B21 = quadB(b, 2), B22 = quadB(b, 3);
    const int m2 = A11.rows, k2 = A11.cols, n2 = d[0].c.cols / 2;
    const ProdTab& T = table(SW_ALGO_WINOGRAD);
    // destinations of product p: every (quadrant, sign) it feeds, within every block of `d`
    auto dest = [&](int p) {
        std::vector<Dest> r;
        for (int t = 0; t < T.ntgt[p]; ++t)
            for (const Dest& x : d) r.push_back(Dest{quad(x.c, T.tgt[p][t].q), x.sign * (float)T.tgt[p][t].s, -1});
        return r;
    };
    const size_t mark = ws_top;
    View X = talloc(m2, k2);
    View Y = tallocB(k2, n2);
    bool ok = true;
    if (L == 1 && bf && !x3 && eb == 4 && k2 > 0) {
        // split-BF16 leaves: every sum a leaf reads gets its bf16 halves from the sum launch itself
        // (no split pass over X or Y); the halves live only while their leaf needs them, so the
        // workspace peak stays at X, Y and one leaf's four halves
        auto leaf = [&](View av, const View* ah, const View* al, View bv, const View* bh, const View* bl,
                        std::vector<Dest> ds) {
            resolve_modes(ds);
            if (ds[0].c.rows <= 0 || ds[0].c.cols <= 0) return true;
            const size_t mk = ws_top;
            View a_h, a_l, b_h, b_l;
            if (ah) { a_h = *ah; a_l = *al; } else split(av, a_h, a_l);
            if (bh) { b_h = *bh; b_l = *bl; } else split(bv, b_h, b_l);
            const bool r = gemm_split_halves(av, a_h, a_l, b_h, b_l, ds);
            ws_top = mk;
            return r;
        };
        const size_t mh = ws_top;
        const View Xh = talloc_half(X.rows, X.cols), Xl = talloc_half(X.rows, X.cols);
        const size_t mx = ws_top;
        const View Yh = talloc_half(Y.rows, Y.cols), Yl = talloc_half(Y.rows, Y.cols);
        add2(X, A11, A21, -1, Y, B22, B12, -1, &Xh, &Xl, &Yh, &Yl);        //  1,  2  S3, T3
        ok &= leaf(X, &Xh, &Xl, Y, &Yh, &Yl, dest(6));                      //  3      P7
        add2(X, A21, A22, +1, Y, B12, B11, -1, &Xh, &Xl, &Yh, &Yl);        //  4,  5  S1, T1
        ok &= leaf(X, &Xh, &Xl, Y, &Yh, &Yl, dest(4));                      //  6      P5
        add2(X, X, A11, -1, Y, B22, Y, -1, &Xh, &Xl, &Yh, &Yl);            //  7,  8  S2, T2
        ok &= leaf(X, &Xh, &Xl, Y, &Yh, &Yl, dest(5));                      //  9      P6
        ws_top = mx;                                                        // (T2's halves done)
        add_split(X, A12, X, -1, Xh, Xl);                                   // 10      S4
        ok &= leaf(X, &Xh, &Xl, B22, nullptr, nullptr, dest(2));            // 11      P3
        ws_top = mh;
        ok &= leaf(A11, nullptr, nullptr, B11, nullptr, nullptr, dest(0));  // 12      P1
        const View Yh4 = talloc_half(Y.rows, Y.cols), Yl4 = talloc_half(Y.rows, Y.cols);
        add_split(Y, Y, B21, -1, Yh4, Yl4);                                 // 18      T4
        ok &= leaf(A22, nullptr, nullptr, Y, &Yh4, &Yl4, dest(3));          // 19      P4
        ws_top = mh;
        ok &= leaf(A12, nullptr, nullptr, B21, nullptr, nullptr, dest(1));  // 21      P2
        ws_top = mark;
        return ok;
    }
    add2(X, A11, A21, -1, Y, B22, B12, -1);         //  1,  2  S3 -> X, T3 -> Y
    ok &= two_temp_folded(X, Y, dest(6), L - 1);    //  3      P7 = S3 T3
    add2(X, A21, A22, +1, Y, B12, B11, -1);         //  4,  5  S1 -> X, T1 -> Y
    ok &= two_temp_folded(X, Y, dest(4), L - 1);    //  6      P5 = S1 T1
    add2(X, X, A11, -1, Y, B22, Y, -1);             //  7,  8  S2 -> X, T2 -> Y
    ok &= two_temp_folded(X, Y, dest(5), L - 1);    //  9      P6 = S2 T2
    add(X, A12, X, -1);                             // 10      S4 -> X
    ok &= two_temp_folded(X, B22, dest(2), L - 1);  // 11      P3 = S4 B22
    ok &= two_temp_folded(A11, B11, dest(0), L - 1);// 12      P1 = A11 B11 (13-17 in its epilogues)
    add(Y, Y, B21, -1);                             // 18      T4 -> Y
    ok &= two_temp_folded(A22, Y, dest(3), L - 1);  // 19      P4 = A22 T4 (20: U6 = U3 - P4)
    ok &= two_temp_folded(A12, B21, dest(1), L - 1);// 21      P2 = A12 B21 (22: U1 = P1 + P2)
    ws_top = mark;
    return ok;
}

// Table 3 (Sec. 3.3): temporaries stored in the quadrants of A, B and C.  Sub-products
// recurse in place too, so each one may overwrite its two operand blocks; the table's
// order never reads a block after such a product consumed it.  Square only: the C22
// quadrant holds the B-side values T1 and T4 (held transposed like every B-side value).
bool Planner::in_place(View a, View b, View c, int L) {
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

int resolve_depth(int m, int n, int k, int cutoff, uint32_t variant, int eb) {
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
sw_status build_plan(sw_handle h, int eb, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                            int m, int n, int k, int cutoff, uint32_t variant, bool dry, Plan* plan,
                            char* ws_base, bool server, uint32_t top_mask, int b_sums_mode, char* b_sums) {
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
    P.top_mask = top_mask;
    P.b_sums_mode = b_sums_mode;
    P.b_sums = b_sums;
    if (server && eb == 4 && !bf) P.force_bn = 256;
    const int L = resolve_depth(m, n, k, cutoff, variant, eb);
    plan->depth = L;
    if (top_mask != 0x7Fu && (sched != SW_SCHED_FUSED || algo == SW_ALGO_NAIVE || L < 1 || L > 3))
        return fail(h, SW_EUNSUPPORTED, "product subsets need a FUSED recursion of depth 1 to 3");

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
        if (top_mask != 0x7Fu && (L == 0 || algo == SW_ALGO_NAIVE || L > 3 || sched != SW_SCHED_FUSED))
            return fail(h, SW_EUNSUPPORTED, "product subsets need a FUSED recursion of depth 1 to 3");
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

sw_status build_batched_plan(sw_handle h, int count, const sw_problem* probs, int cutoff, uint32_t variant,
                                    bool dry, Plan* plan, int bn, bool pair, bool pack) {
    Planner P;
    P.batch_bn = bn;
    P.batch_pair = pair;
    P.pack_in_gemm = pack;
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

}  // namespace swh
