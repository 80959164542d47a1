/*
 * oracle.c -- plain, slow, FP64 CPU reference for the Strassen / Strassen-Winograd
 * matrix product (arXiv 2309.00628, "Algoritmos para Multiplicacao Matricial").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may call, link or load this file.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Conventions.  Sec. 2.1 writes A m x n, B n x k and reuses k as the loop index;
 * Sec. 3.4 writes A m x k, B k x n.  We follow Sec. 3.4 (BLAS naming):
 *   C (m x n) = A (m x k) * B (k x n), row-major, with leading dimensions.
 *   Quadrants are X11 X12 / X21 X22.
 *
 * Recursion depth.  Alg. 2 and Alg. 3 recurse down to the 1x1 product; Sec. 3.4
 * stops at a cutoff and calls the naive method (Alg. 1) there.  Reading used
 * here: recurse while min(m, n, k) > cutoff, with cutoff >= 1 (cutoff 1 is the
 * literal 1x1 base case).
 *
 * Odd sizes (Sec. 3.1).  The paper pads with zero rows/columns and leaves other
 * methods unspecified.  Two readings are provided:
 *   ORC_PAD  : pad once, up front, so every dimension is a multiple of 2^L
 *              (L = depth from the cutoff rule), then halve exactly L times.
 *   ORC_PEEL : at each level peel an odd last row / column / inner index, recurse
 *              on the even part and fix the peeled part up with naive products.
 *
 * Floating point: IEEE binary64, round to nearest.  The naive product sums with the
 * inner index ascending, as Alg. 1 does.
 *
 * Parity status: every public function is pinned by the CPU tests in
 * tests/test_oracle_pins.py -- the hand-worked 2x2 values of each form, identity
 * and permutation matrices, integer bit-exactness against the naive product,
 * brute force on tiny sizes, the cutoff inequality in closed form, and the
 * schedules' liveness shadow.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PAD 0
#define ORC_PEEL 1

enum { ALG_STRASSEN = 0, ALG_WINOGRAD = 1, ALG_KNUTH = 2, ALG_TWO_TEMP = 3, ALG_IN_PLACE = 4 };

/* A strided view of a row-major matrix. */
typedef struct {
    double *p;
    long rows, cols, ld;
} mat;

static mat view(double *p, long rows, long cols, long ld) {
    mat v = {p, rows, cols, ld};
    return v;
}

static mat sub(mat a, long r0, long c0, long rows, long cols) {
    return view(a.p + r0 * a.ld + c0, rows, cols, a.ld);
}

/* quadrant q in {0:X11, 1:X12, 2:X21, 3:X22} of a matrix with even dims */
static mat quad(mat a, int q) {
    long h = a.rows / 2, w = a.cols / 2;
    return sub(a, (q >> 1) * h, (q & 1) * w, h, w);
}

static mat alloc_mat(long rows, long cols) {
    size_t r = (size_t)(rows > 0 ? rows : 1), c = (size_t)(cols > 0 ? cols : 1);
    double *p = (double *)calloc(r * c, sizeof(double));
    return view(p, rows, cols, cols);
}

static void free_mat(mat a) { free(a.p); }

static void copy_into(mat dst, mat src) {
    for (long i = 0; i < src.rows; ++i)
        memcpy(dst.p + i * dst.ld, src.p + i * src.ld, (size_t)src.cols * sizeof(double));
}

/* Z = X + s*Y elementwise, s = +1 or -1: the block additions of Sec. 2.2 / 2.3. */
static void addsub(mat z, mat x, mat y, double s) {
    for (long i = 0; i < z.rows; ++i)
        for (long j = 0; j < z.cols; ++j)
            z.p[i * z.ld + j] = x.p[i * x.ld + j] + s * y.p[i * y.ld + j];
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 (Sec. 2.1): c_ij = sum_p a_ip b_pj, p ascending.                    */
/* ------------------------------------------------------------------------- */
static void naive(mat a, mat b, mat c) {
    for (long i = 0; i < c.rows; ++i)
        for (long j = 0; j < c.cols; ++j) {
            double s = 0.0;
            for (long p = 0; p < a.cols; ++p) s += a.p[i * a.ld + p] * b.p[p * b.ld + j];
            c.p[i * c.ld + j] = s;
        }
}

int orc_naive(long m, long n, long k, const double *A, long lda, const double *B, long ldb,
              double *C, long ldc) {
    if (m < 0 || n < 0 || k < 0) return 1;
    naive(view((double *)A, m, k, lda), view((double *)B, k, n, ldb), view(C, m, n, ldc));
    return 0;
}

/* Same arithmetic as orc_naive (identical per-element summation order), with the
 * rows spread over host threads.  Only used to time the oracle on all cores. */
int orc_naive_mt(long m, long n, long k, const double *A, long lda, const double *B, long ldb,
                 double *C, long ldc, int threads) {
    if (m < 0 || n < 0 || k < 0) return 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long i = 0; i < m; ++i)
        for (long j = 0; j < n; ++j) {
            double s = 0.0;
            for (long p = 0; p < k; ++p) s += A[i * lda + p] * B[p * ldb + j];
            C[i * ldc + j] = s;
        }
    return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Depth from the cutoff (Sec. 3.4, reading above): halve while               */
/* min(ceil(m/2^l), ceil(n/2^l), ceil(k/2^l)) > cutoff.                       */
/* ------------------------------------------------------------------------- */
int orc_depth(long m, long n, long k, long cutoff) {
    if (cutoff < 1) cutoff = 1;
    int L = 0;
    while (L < 40) {
        long s = 1L << L;
        long mm = (m + s - 1) / s, nn = (n + s - 1) / s, kk = (k + s - 1) / s;
        long lo = mm < nn ? mm : nn;
        if (kk < lo) lo = kk;
        if (lo > cutoff) ++L; else break;
    }
    return L;
}

/* Sec. 3.4 cost model.  M(m,k,n) = multiplications + additions of the naive
 * product = mkn + mn(k-1); G(r,c) = rc for one block addition.  Returns
 * lhs = M(m,k,n) and rhs = 7M(m/2,k/2,n/2) + 4G(m/2,k/2) + 4G(k/2,n/2) + 7G(m/2,n/2)
 * (one recursion level with 15 block additions), both in exact doubles. */
void orc_cutoff_model(double m, double k, double n, double *lhs, double *rhs) {
    double M = m * k * n + m * n * (k - 1.0);
    double m2 = m / 2, k2 = k / 2, n2 = n / 2;
    double M2 = m2 * k2 * n2 + m2 * n2 * (k2 - 1.0);
    *lhs = M;
    *rhs = 7.0 * M2 + 4.0 * (m2 * k2) + 4.0 * (k2 * n2) + 7.0 * (m2 * n2);
}

/* ------------------------------------------------------------------------- */
/* Sub-product dispatch.  Each algorithm below is written as ONE recursion     */
/* level; its sub-products go through product(), which either recurses with   */
/* one level fewer (PAD) or peels and re-checks the cutoff (PEEL).             */
/* ------------------------------------------------------------------------- */
typedef struct ctx ctx;
typedef void (*level_fn)(mat a, mat b, mat c, ctx *x, int top);
struct ctx {
    level_fn level;
    int mode;     /* ORC_PAD / ORC_PEEL */
    int L;        /* PAD: levels still to do */
    long cutoff;  /* PEEL */
    int destroys; /* the level overwrites its A/B operands (in-place schedule) */
};

static double *g_trace = NULL; /* top-level intermediates, element [0][0] */
static int g_sched_error = 0;  /* set when a schedule's shadow finds a dead read */
/* Products of the TOP level that take part (bit i: the (i+1)-th product of Sec. 2.2 / 2.3 in
 * the numbering of strassen_level / winograd_level; Knuth's form uses the BDPZ numbering).  A
 * product outside the mask is taken as the zero block and the level's post-additions run as
 * written: C then holds the top-level products' contributions to C restricted to the mask. */
static unsigned g_top_mask = 0x7Fu;

static void tr(int idx, mat x) {
    if (g_trace && x.rows > 0 && x.cols > 0) g_trace[idx] = x.p[0];
}

static void product_at(mat a, mat b, mat c, ctx *x, int top);

static void product(mat a, mat b, mat c, ctx *x) { product_at(a, b, c, x, 0); }

static void zero_mat(mat c) {
    for (long i = 0; i < c.rows; ++i)
        for (long j = 0; j < c.cols; ++j) c.p[i * c.ld + j] = 0.0;
}

/* Sub-product `idx` of a level: at the top level a product outside g_top_mask is the zero block. */
static void product_top(mat a, mat b, mat c, ctx *x, int top, int idx) {
    if (top && !((g_top_mask >> idx) & 1u)) { zero_mat(c); return; }
    product(a, b, c, x);
}

static void product_at(mat a, mat b, mat c, ctx *x, int top) {
    if (x->mode == ORC_PAD) {
        if (x->L == 0) { naive(a, b, c); return; }
        x->L--;
        x->level(a, b, c, x, top);
        x->L++;
        return;
    }
    long m = a.rows, k = a.cols, n = b.cols;
    long lo = m < n ? m : n;
    if (k < lo) lo = k;
    if (lo <= x->cutoff || lo < 2) { naive(a, b, c); return; }
    long me = m & ~1L, ne = n & ~1L, ke = k & ~1L;
    /* Edge fixups first: they read the even parts of A and B, which the in-place
     * schedule overwrites. */
    if (m & 1) naive(sub(a, m - 1, 0, 1, k), b, sub(c, m - 1, 0, 1, n));
    if (n & 1) naive(sub(a, 0, 0, me, k), sub(b, 0, n - 1, k, 1), sub(c, 0, n - 1, me, 1));
    x->level(sub(a, 0, 0, me, ke), sub(b, 0, 0, ke, ne), sub(c, 0, 0, me, ne), x, top);
    if (k & 1) /* rank-1 update with the peeled inner index (not part of the even blocks) */
        for (long i = 0; i < me; ++i)
            for (long j = 0; j < ne; ++j)
                c.p[i * c.ld + j] += a.p[i * a.ld + (k - 1)] * b.p[(k - 1) * b.ld + j];
}

/* ------------------------------------------------------------------------- */
/* Strassen, Sec. 2.2 / Alg. 2:                                               */
/*   P1=(A11+A22)(B11+B22)  P2=(A21+A22)B11  P3=A11(B12-B22)  P4=A22(-B11+B21) */
/*   P5=(A11+A12)B22  P6=(-A11+A21)(B11+B12)  P7=(A12-A22)(B21+B22)            */
/*   C11=P1+P4-P5+P7  C12=P3+P5  C21=P2+P4  C22=P1+P3-P2+P6 (left to right)    */
/* trace slots 0..6 = P1..P7                                                   */
/* ------------------------------------------------------------------------- */
static void strassen_level(mat a, mat b, mat c, ctx *x, int top) {
    mat A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
    mat B11 = quad(b, 0), B12 = quad(b, 1), B21 = quad(b, 2), B22 = quad(b, 3);
    long m2 = A11.rows, k2 = A11.cols, n2 = B11.cols;
    mat sa = alloc_mat(m2, k2), sb = alloc_mat(k2, n2), P[7];
    for (int i = 0; i < 7; ++i) P[i] = alloc_mat(m2, n2);
    addsub(sa, A11, A22, +1); addsub(sb, B11, B22, +1); product_top(sa, sb, P[0], x, top, 0);
    addsub(sa, A21, A22, +1); product_top(sa, B11, P[1], x, top, 1);
    addsub(sb, B12, B22, -1); product_top(A11, sb, P[2], x, top, 2);
    addsub(sb, B21, B11, -1); product_top(A22, sb, P[3], x, top, 3);
    addsub(sa, A11, A12, +1); product_top(sa, B22, P[4], x, top, 4);
    addsub(sa, A21, A11, -1); addsub(sb, B11, B12, +1); product_top(sa, sb, P[5], x, top, 5);
    addsub(sa, A12, A22, -1); addsub(sb, B21, B22, +1); product_top(sa, sb, P[6], x, top, 6);
    if (top) for (int i = 0; i < 7; ++i) tr(i, P[i]);
    mat C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
    addsub(C11, P[0], P[3], +1); addsub(C11, C11, P[4], -1); addsub(C11, C11, P[6], +1);
    addsub(C12, P[2], P[4], +1);
    addsub(C21, P[1], P[3], +1);
    addsub(C22, P[0], P[2], +1); addsub(C22, C22, P[1], -1); addsub(C22, C22, P[5], +1);
    for (int i = 0; i < 7; ++i) free_mat(P[i]);
    free_mat(sa); free_mat(sb);
}

/* ------------------------------------------------------------------------- */
/* Strassen-Winograd, Boyer-Dumas-Pernet-Zhou 22-operation form (Sec. 2.3),   */
/* allocating every temporary as Alg. 3 does:                                 */
/*   S1=A21+A22 S2=S1-A11 S3=A11-A21 T1=B12-B11 T2=B22-T1 T3=B22-B12           */
/*   S4=A12-S2 T4=T2-B21                                                       */
/*   P1=A11B11 P2=A12B21 P3=S4B22 P4=A22T4 P5=S1T1 P6=S2T2 P7=S3T3              */
/*   U1=P1+P2 U2=P1+P6 U3=U2+P7 U4=U2+P5 U5=U4+P3 U6=U3-P4 U7=U3+P5            */
/*   C = [U1 U5; U6 U7]                                                        */
/* trace slots 8..11 S1..S4, 12..15 T1..T4, 16..22 P1..P7, 23..29 U1..U7       */
/* (the value numbering of the schedule tables below).                        */
/* ------------------------------------------------------------------------- */
static void winograd_level(mat a, mat b, mat c, ctx *x, int top) {
    mat A11 = quad(a, 0), A12 = quad(a, 1), A21 = quad(a, 2), A22 = quad(a, 3);
    mat B11 = quad(b, 0), B12 = quad(b, 1), B21 = quad(b, 2), B22 = quad(b, 3);
    long m2 = A11.rows, k2 = A11.cols, n2 = B11.cols;
    mat S[4], T[4], P[7];
    for (int i = 0; i < 4; ++i) { S[i] = alloc_mat(m2, k2); T[i] = alloc_mat(k2, n2); }
    for (int i = 0; i < 7; ++i) P[i] = alloc_mat(m2, n2);
    addsub(S[0], A21, A22, +1);
    addsub(S[1], S[0], A11, -1);
    addsub(S[2], A11, A21, -1);
    addsub(T[0], B12, B11, -1);
    addsub(T[1], B22, T[0], -1);
    addsub(T[2], B22, B12, -1);
    addsub(S[3], A12, S[1], -1);
    addsub(T[3], T[1], B21, -1);
    product_top(A11, B11, P[0], x, top, 0);
    product_top(A12, B21, P[1], x, top, 1);
    product_top(S[3], B22, P[2], x, top, 2);
    product_top(A22, T[3], P[3], x, top, 3);
    product_top(S[0], T[0], P[4], x, top, 4);
    product_top(S[1], T[1], P[5], x, top, 5);
    product_top(S[2], T[2], P[6], x, top, 6);
    if (top) {
        for (int i = 0; i < 4; ++i) { tr(8 + i, S[i]); tr(12 + i, T[i]); }
        for (int i = 0; i < 7; ++i) tr(16 + i, P[i]);
    }
    /* The U chain reuses the P temporaries once their products are consumed:
     * U2 -> P6's block, U3 -> P7's, U4 -> P1's (P1 is last read by U1 and U2). */
    mat C11 = quad(c, 0), C12 = quad(c, 1), C21 = quad(c, 2), C22 = quad(c, 3);
    addsub(C11, P[0], P[1], +1);  /* U1 = P1 + P2 */
    addsub(P[5], P[0], P[5], +1); /* U2 = P1 + P6 */
    addsub(P[6], P[5], P[6], +1); /* U3 = U2 + P7 */
    addsub(P[0], P[5], P[4], +1); /* U4 = U2 + P5 */
    addsub(C12, P[0], P[2], +1);  /* U5 = U4 + P3 */
    addsub(C21, P[6], P[3], -1);  /* U6 = U3 - P4 */
    addsub(C22, P[6], P[4], +1);  /* U7 = U3 + P5 */
    if (top) {
        tr(23, C11); tr(24, P[5]); tr(25, P[6]); tr(26, P[0]); tr(27, C12); tr(28, C21); tr(29, C22);
    }
    for (int i = 0; i < 4; ++i) { free_mat(S[i]); free_mat(T[i]); }
    for (int i = 0; i < 7; ++i) free_mat(P[i]);
}

/* ------------------------------------------------------------------------- */
/* Strassen-Winograd in Knuth's form (Sec. 2.3, first bullet):               */
/*   [a b; c d][A C; B D] = [aA+bB, w+v+(a+b-c-d)D; w+u+d(B+C-A-D), w+u+v]      */
/*   u=(c-a)(C-D)  v=(c+d)(C-A)  w=aA+(c+d-a)(A+D-C)                            */
/* with a,b,c,d = A11,A12,A21,A22 and A,C,B,D = B11,B12,B21,B22.                */
/* trace slots 0 u, 1 v, 2 w, 3 aA, 4 bB, 5 (a+b-c-d)D, 6 d(B+C-A-D)           */
/* ------------------------------------------------------------------------- */
static void knuth_level(mat X, mat Y, mat Z, ctx *x, int top) {
    mat a = quad(X, 0), b = quad(X, 1), c = quad(X, 2), d = quad(X, 3);
    mat A = quad(Y, 0), C = quad(Y, 1), B = quad(Y, 2), D = quad(Y, 3);
    long m2 = a.rows, k2 = a.cols, n2 = A.cols;
    mat l = alloc_mat(m2, k2), r = alloc_mat(k2, n2);
    mat u = alloc_mat(m2, n2), v = alloc_mat(m2, n2), w = alloc_mat(m2, n2);
    mat aA = alloc_mat(m2, n2), bB = alloc_mat(m2, n2), t = alloc_mat(m2, n2);
    addsub(l, c, a, -1); addsub(r, C, D, -1); product_top(l, r, u, x, top, 6);
    addsub(l, c, d, +1); addsub(r, C, A, -1); product_top(l, r, v, x, top, 4);
    product_top(a, A, aA, x, top, 0);
    addsub(l, c, d, +1); addsub(l, l, a, -1);
    addsub(r, A, D, +1); addsub(r, r, C, -1);
    product_top(l, r, t, x, top, 5); addsub(w, aA, t, +1);
    product_top(b, B, bB, x, top, 1);
    mat z11 = quad(Z, 0), z12 = quad(Z, 1), z21 = quad(Z, 2), z22 = quad(Z, 3);
    addsub(z11, aA, bB, +1);
    if (top) { tr(0, u); tr(1, v); tr(2, w); tr(3, aA); tr(4, bB); }
    addsub(l, a, b, +1); addsub(l, l, c, -1); addsub(l, l, d, -1);
    product_top(l, D, t, x, top, 2);
    if (top) tr(5, t);
    addsub(z12, w, v, +1); addsub(z12, z12, t, +1);
    addsub(r, B, C, +1); addsub(r, r, A, -1); addsub(r, r, D, -1);
    product_top(d, r, t, x, top, 3);
    if (top) tr(6, t);
    addsub(z21, w, u, +1); addsub(z21, z21, t, +1);
    addsub(z22, w, u, +1); addsub(z22, z22, v, +1);
    free_mat(l); free_mat(r); free_mat(u); free_mat(v); free_mat(w);
    free_mat(aA); free_mat(bB); free_mat(t);
}

/* ------------------------------------------------------------------------- */
/* The two low-allocation schedules of Sec. 3.3, executed step by step from   */
/* Table 2 and Table 3.  Slots are quadrant-sized storage; values are the     */
/* blocks of the BDPZ form.  A shadow records which value each slot holds and */
/* every read checks that the value it wants is still live.                  */
/* ------------------------------------------------------------------------- */
enum { sA11, sA12, sA21, sA22, sB11, sB12, sB21, sB22, sC11, sC12, sC21, sC22, sX, sY, NSLOT };
enum {
    vA11, vA12, vA21, vA22, vB11, vB12, vB21, vB22,
    vS1, vS2, vS3, vS4, vT1, vT2, vT3, vT4,
    vP1, vP2, vP3, vP4, vP5, vP6, vP7,
    vU1, vU2, vU3, vU4, vU5, vU6, vU7, vDEAD, NVAL = vDEAD
};
enum { OP_ADD, OP_SUB, OP_MUL };

typedef struct {
    int op;     /* value = v1 (+ | - | x) v2 */
    int val;    /* value produced */
    int dst;    /* slot it is stored in */
    int v1, v2; /* values read */
} step;

/* Table 2, "Two Temp Winograd": temporaries X and Y. */
static const step two_temp_table[22] = {
    {OP_SUB, vS3, sX, vA11, vA21},   {OP_SUB, vT3, sY, vB22, vB12},   {OP_MUL, vP7, sC21, vS3, vT3},
    {OP_ADD, vS1, sX, vA21, vA22},   {OP_SUB, vT1, sY, vB12, vB11},   {OP_MUL, vP5, sC22, vS1, vT1},
    {OP_SUB, vS2, sX, vS1, vA11},    {OP_SUB, vT2, sY, vB22, vT1},    {OP_MUL, vP6, sC12, vS2, vT2},
    {OP_SUB, vS4, sX, vA12, vS2},    {OP_MUL, vP3, sC11, vS4, vB22},  {OP_MUL, vP1, sX, vA11, vB11},
    {OP_ADD, vU2, sC12, vP1, vP6},   {OP_ADD, vU3, sC21, vU2, vP7},   {OP_ADD, vU4, sC12, vU2, vP5},
    {OP_ADD, vU7, sC22, vU3, vP5},   {OP_ADD, vU5, sC12, vU4, vP3},   {OP_SUB, vT4, sY, vT2, vB21},
    {OP_MUL, vP4, sC11, vA22, vT4},  {OP_SUB, vU6, sC21, vU3, vP4},   {OP_MUL, vP2, sC11, vA12, vB21},
    {OP_ADD, vU1, sC11, vP1, vP2},
};

/* Table 3, "In-Place Winograd": temporaries in the quadrants of A, B and C. */
static const step in_place_table[22] = {
    {OP_SUB, vS3, sC11, vA11, vA21}, {OP_ADD, vS1, sA21, vA21, vA22}, {OP_SUB, vT1, sC22, vB12, vB11},
    {OP_SUB, vT3, sB12, vB22, vB12}, {OP_MUL, vP7, sC21, vS3, vT3},   {OP_SUB, vS2, sC12, vS1, vA11},
    {OP_MUL, vP1, sC11, vA11, vB11}, {OP_SUB, vT2, sB11, vB22, vT1},  {OP_MUL, vP5, sA11, vS1, vT1},
    {OP_SUB, vT4, sC22, vT2, vB21},  {OP_MUL, vP4, sA21, vA22, vT4},  {OP_SUB, vS4, sA22, vA12, vS2},
    {OP_MUL, vP6, sC22, vS2, vT2},   {OP_ADD, vU2, sC22, vP1, vP6},   {OP_MUL, vP2, sC12, vA12, vB21},
    {OP_ADD, vU1, sC11, vP1, vP2},   {OP_ADD, vU4, sC12, vU2, vP5},   {OP_ADD, vU3, sC22, vU2, vP7},
    {OP_SUB, vU6, sC21, vU3, vP4},   {OP_ADD, vU7, sC22, vU3, vP5},   {OP_MUL, vP3, sA12, vS4, vB22},
    {OP_ADD, vU5, sC12, vU4, vP3},
};

static const step *g_tables[3] = {two_temp_table, in_place_table, NULL};
static step g_custom_table[22]; /* a caller-supplied table (tests plant mistakes here) */

/* Shape of a value: 'a' (m2 x k2), 'b' (k2 x n2) or 'c' (m2 x n2). */
static char shape_of(int v) {
    if (v <= vA22 || (v >= vS1 && v <= vS4)) return 'a';
    if (v <= vB22 || (v >= vT1 && v <= vT4)) return 'b';
    return 'c';
}

static int slot_of(const int *holds, int v) {
    for (int s = 0; s < NSLOT; ++s)
        if (holds[s] == v) return s;
    return -1;
}

/* View of slot s holding a value of the given shape.  Quadrant slots keep the
 * parent's leading dimension; the X/Y temporaries are dense. */
static mat slot_view(mat *slot, int s, char shape, long m2, long k2, long n2) {
    long r = shape == 'b' ? k2 : m2, c = shape == 'a' ? k2 : n2;
    if (s == sX || s == sY) return view(slot[s].p, r, c, c);
    return view(slot[s].p, r, c, slot[s].ld);
}

static void run_table(const step *tab, mat *slot, int *holds, ctx *x, int top, long m2, long k2,
                      long n2) {
    for (int i = 0; i < 22; ++i) {
        const step *st = &tab[i];
        int s1 = slot_of(holds, st->v1), s2 = slot_of(holds, st->v2);
        if (s1 < 0 || s2 < 0) { g_sched_error = 1; return; }
        mat o1 = slot_view(slot, s1, shape_of(st->v1), m2, k2, n2);
        mat o2 = slot_view(slot, s2, shape_of(st->v2), m2, k2, n2);
        mat d = slot_view(slot, st->dst, shape_of(st->val), m2, k2, n2);
        if (st->op == OP_MUL) {
            product(o1, o2, d, x);
            if (x->destroys) { /* an in-place sub-product may overwrite its operands */
                if (s1 != st->dst) holds[s1] = vDEAD;
                if (s2 != st->dst) holds[s2] = vDEAD;
            }
        } else {
            addsub(d, o1, o2, st->op == OP_ADD ? +1.0 : -1.0);
        }
        holds[st->dst] = st->val;
        if (top) tr(st->val, d);
    }
    if (holds[sC11] != vU1 || holds[sC12] != vU5 || holds[sC21] != vU6 || holds[sC22] != vU7)
        g_sched_error = 1;
}

static void schedule_level(mat a, mat b, mat c, ctx *x, int top, int which) {
    mat slot[NSLOT];
    int holds[NSLOT];
    for (int q = 0; q < 4; ++q) {
        slot[sA11 + q] = quad(a, q); slot[sB11 + q] = quad(b, q); slot[sC11 + q] = quad(c, q);
        holds[sA11 + q] = vA11 + q; holds[sB11 + q] = vB11 + q; holds[sC11 + q] = vDEAD;
    }
    long m2 = a.rows / 2, k2 = a.cols / 2, n2 = b.cols / 2;
    double *xp = NULL, *yp = NULL;
    if (which == 0 || which == 3) { /* Table 2, or a caller's table under its rules */
        /* X holds A-quadrant sums (m2 x k2) and P1 (m2 x n2): sized for the larger. */
        long xs = m2 * (k2 > n2 ? k2 : n2);
        xp = (double *)calloc((size_t)(xs > 0 ? xs : 1), sizeof(double));
        yp = (double *)calloc((size_t)(k2 * n2 > 0 ? k2 * n2 : 1), sizeof(double));
    }
    slot[sX] = view(xp, 0, 0, 0); slot[sY] = view(yp, 0, 0, 0);
    holds[sX] = vDEAD; holds[sY] = vDEAD;
    run_table(which == 3 ? g_custom_table : g_tables[which], slot, holds, x, top, m2, k2, n2);
    free(xp); free(yp);
}

static void two_temp_level(mat a, mat b, mat c, ctx *x, int top) { schedule_level(a, b, c, x, top, 0); }
static void in_place_level(mat a, mat b, mat c, ctx *x, int top) { schedule_level(a, b, c, x, top, 1); }
static void custom_level(mat a, mat b, mat c, ctx *x, int top) { schedule_level(a, b, c, x, top, 2); }
static void custom_tt_level(mat a, mat b, mat c, ctx *x, int top) { schedule_level(a, b, c, x, top, 3); }

/* Copy table `which` (0 two-temp, 1 in-place) out as 22 x {op, val, dst, v1, v2}. */
int orc_schedule_table(int which, int *out) {
    if (which < 0 || which > 1) return 1;
    for (int i = 0; i < 22; ++i) {
        const step *st = &g_tables[which][i];
        out[5 * i + 0] = st->op; out[5 * i + 1] = st->val; out[5 * i + 2] = st->dst;
        out[5 * i + 3] = st->v1; out[5 * i + 4] = st->v2;
    }
    return 0;
}

static const level_fn g_levels[7] = {strassen_level, winograd_level, knuth_level, two_temp_level,
                                     in_place_level, custom_level, custom_tt_level};

/* ------------------------------------------------------------------------- */
/* Public recursive entry.  alg: 0 Strassen, 1 Winograd (BDPZ, allocating),   */
/* 2 Winograd (Knuth form), 3 Two-Temp schedule, 4 In-Place schedule.         */
/* In-place needs m == n == k and OVERWRITES A and B (pass copies).           */
/* trace: if non-NULL, receives top-level intermediates (see slot lists).     */
/* Returns 0 on success, 1 on bad arguments, 2 if a schedule's shadow failed. */
/* ------------------------------------------------------------------------- */
int orc_recursive(int alg, long m, long n, long k, double *A, long lda, double *B, long ldb,
                  double *C, long ldc, long cutoff, int mode, double *trace) {
    if (alg < 0 || alg > 6 || m < 0 || n < 0 || k < 0) return 1;
    if ((alg == ALG_IN_PLACE || alg == 5) && !(m == n && n == k)) return 1;
    if (cutoff < 1) cutoff = 1;
    ctx x;
    x.level = g_levels[alg];
    x.mode = mode;
    x.cutoff = cutoff;
    x.destroys = alg == ALG_IN_PLACE || alg == 5;
    g_trace = trace;
    g_sched_error = 0;
    mat a = view(A, m, k, lda), b = view(B, k, n, ldb), c = view(C, m, n, ldc);
    if (m == 0 || n == 0) { g_trace = NULL; return 0; }
    if (mode == ORC_PEEL) {
        x.L = 0;
        product_at(a, b, c, &x, 1);
    } else {
        int L = orc_depth(m, n, k, cutoff);
        long s = 1L << L;
        long mp = (m + s - 1) / s * s, np = (n + s - 1) / s * s, kp = (k + s - 1) / s * s;
        x.L = L;
        if (mp == m && np == n && kp == k) {
            product_at(a, b, c, &x, 1);
        } else {
            mat ap = alloc_mat(mp, kp), bp = alloc_mat(kp, np), cp = alloc_mat(mp, np);
            copy_into(ap, a); copy_into(bp, b);
            product_at(ap, bp, cp, &x, 1);
            copy_into(c, sub(cp, 0, 0, m, n));
            if (x.destroys) { copy_into(a, sub(ap, 0, 0, m, k)); copy_into(b, sub(bp, 0, 0, k, n)); }
            free_mat(ap); free_mat(bp); free_mat(cp);
        }
    }
    g_trace = NULL;
    return g_sched_error ? 2 : 0;
}

/* The top-level products in `mask` only (bit i = the (i+1)-th product of the level; Knuth's form
 * in the BDPZ numbering): C receives their contributions to C, the other products taken as zero
 * blocks (alg 0 Strassen, 1 Winograd BDPZ, 2 Knuth; PAD; depth >= 1).  Summing the results of
 * masks that partition the seven products gives the product of orc_recursive, up to the order of
 * the floating-point additions.  Returns 1 on bad arguments or depth 0. */
int orc_recursive_products(int alg, long m, long n, long k, double *A, long lda, double *B, long ldb,
                           double *C, long ldc, long cutoff, unsigned mask) {
    if (alg < 0 || alg > 2 || (mask & ~0x7Fu) != 0) return 1;
    if (orc_depth(m, n, k, cutoff < 1 ? 1 : cutoff) < 1) return 1;
    g_top_mask = mask;
    int rc = orc_recursive(alg, m, n, k, A, lda, B, ldb, C, ldc, cutoff, ORC_PAD, NULL);
    g_top_mask = 0x7Fu;
    return rc;
}

/* Run a caller-supplied 22-step table (same encoding as orc_schedule_table) with
 * the rules of Table 3 (rules 0: in place, square only, operands of sub-products are
 * destroyed) or of Table 2 (rules 1: the X and Y temporaries, any shape, operands kept).
 * Lets the tests plant a mistake in a copy of Table 2 or 3 and watch the shadow catch it. */
int orc_recursive_table(const int *tab, int rules, long m, long n, long k, double *A, double *B,
                        double *C, long cutoff, double *trace) {
    for (int i = 0; i < 22; ++i) {
        g_custom_table[i].op = tab[5 * i + 0]; g_custom_table[i].val = tab[5 * i + 1];
        g_custom_table[i].dst = tab[5 * i + 2]; g_custom_table[i].v1 = tab[5 * i + 3];
        g_custom_table[i].v2 = tab[5 * i + 4];
        if (g_custom_table[i].dst < 0 || g_custom_table[i].dst >= NSLOT) return 1;
    }
    g_tables[2] = g_custom_table;
    if (rules == 1) return orc_recursive(6, m, n, k, A, k, B, n, C, n, cutoff, ORC_PAD, trace);
    if (!(m == n && n == k)) return 1;
    return orc_recursive(5, n, n, n, A, n, B, n, C, n, cutoff, ORC_PAD, trace);
}

/* Peak number of temporary elements held at once, depth L, even splits:
 *   sched 0 -- the allocating recursion (Alg. 3): 15 temporaries per level
 *              (4 S, 4 T, 7 P; the U chain reuses the P blocks), all levels live;
 *   sched 1 -- the two-temp schedule (Table 2): X = m2 max(k2, n2), Y = k2 n2
 *              per level, all levels live.
 * Pure counting, used to pin the workspace accounting. */
double orc_workspace_elems(int sched, long m, long n, long k, int L) {
    double tot = 0.0;
    double mm = (double)m, nn = (double)n, kk = (double)k;
    for (int l = 0; l < L; ++l) {
        mm /= 2; nn /= 2; kk /= 2;
        if (sched == 0) /* allocating BDPZ */
            tot += 4 * mm * kk + 4 * kk * nn + 7 * mm * nn;
        else if (sched == 1) /* two temp: X = max(m2 k2, m2 n2), Y = k2 n2 */
            tot += (mm * (kk > nn ? kk : nn)) + kk * nn;
    }
    return tot;
}

/* max|C - R| / (k * max|A| * max|B|): the normalised error of the tests. */
double orc_err_norm(long m, long n, long k, const double *C, long ldc, const double *R, long ldr,
                    const double *A, long lda, const double *B, long ldb) {
    double e = 0.0, am = 0.0, bm = 0.0;
    for (long i = 0; i < m; ++i)
        for (long j = 0; j < n; ++j) {
            double d = fabs(C[i * ldc + j] - R[i * ldr + j]);
            if (d > e || d != d) e = d;
        }
    for (long i = 0; i < m; ++i)
        for (long p = 0; p < k; ++p) am = fmax(am, fabs(A[i * lda + p]));
    for (long p = 0; p < k; ++p)
        for (long j = 0; j < n; ++j) bm = fmax(bm, fabs(B[p * ldb + j]));
    double den = (double)(k > 0 ? k : 1) * am * bm;
    if (den == 0.0) return e;
    return e / den;
}
