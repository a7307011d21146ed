/*
 * CPU oracle for the MoA generalized inner and outer product
 * (Raynolds & Mullin, "A generalized inner and outer product of arbitrary
 * multi-dimensional arrays using A Mathematics of Arrays (MoA)").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only tests/, __graft_entry__.smoke() and the cpu_baseline
 * / reference arm of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library: it is the plain, slow definition of what the
 * library computes, written so it can be checked against the paper by eye.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction, no flush-to-zero), so every floating operation below
 * is one IEEE-754 binary64 operation in program order.
 *
 * Conventions (the paper's statement of the problem, Sec. I):
 *  - an array is a shape vector (rho A) plus an element vector;
 *  - elements are stored contiguously in row-major order (the appendix
 *    addresses row i of the left operand, row p of the right operand and
 *    row i of the result at multiples of their row lengths);
 *  - psi-indexing: a full index vector idx selects the element at
 *    offset sum_k idx[k] * prod_{m>k} rho[m].
 *
 * Operator codes (the oracle's own, mapped by oracle/__init__.py):
 *   0 add, 1 sub, 2 mul, 3 div, 4 min, 5 max, 6 or, 7 and.
 * Output kinds for the floating outer product: 0 f64, 1 f32, 2 bf16 bits.
 *
 * Pins: every function below is checked in tests/test_oracle.py against a
 * library routine (numpy tensordot / ufunc.outer / matmul, torch's bf16 cast),
 * exact rational arithmetic (fractions.Fraction), closed forms (identity and
 * all-ones operands), hand-computed shortest paths (tests/golden/), or the
 * identity "inner = reduce of the outer product along the matched axes".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OP_ADD = 0, OP_SUB = 1, OP_MUL = 2, OP_DIV = 3, OP_MIN = 4, OP_MAX = 5, OP_OR = 6, OP_AND = 7 };
enum { ORC_OK = 0, ORC_ERR_RANK = 1, ORC_ERR_SHAPE = 2, ORC_ERR_OP = 3, ORC_ERR_INDEX = 4 };

#define MAXRANK 16

/* ------------------------------------------------------------------ psi */

/* Number of elements: the product of the shape vector (1 for rank 0). */
static int64_t tau(int rank, const int64_t *rho) {
    int64_t n = 1;
    for (int k = 0; k < rank; ++k) n *= rho[k];
    return n;
}

/* Row-major offset of the element selected by a full index vector (psi). */
static int64_t psi_offset(int rank, const int64_t *rho, const int64_t *idx) {
    int64_t off = 0;
    for (int k = 0; k < rank; ++k) off = off * rho[k] + idx[k];
    return off;
}

/* Inverse of psi_offset: the index vector of the element at a flat offset. */
static void psi_index(int64_t flat, int rank, const int64_t *rho, int64_t *idx) {
    for (int k = rank - 1; k >= 0; --k) {
        idx[k] = rho[k] ? flat % rho[k] : 0;
        flat = rho[k] ? flat / rho[k] : 0;
    }
}

int oracle_inner_shape(int rankA, const int64_t *shA, int rankB, const int64_t *shB, int *rankD, int64_t *shD) {
    /* Eq. (2): D_{ijklm} = sum_p A_{ijkp} B_{plm}; the last axis of A meets
     * the first axis of B and both disappear from the result. */
    if (rankA < 1 || rankB < 1 || rankA + rankB - 2 > MAXRANK) return ORC_ERR_RANK;
    if (shA[rankA - 1] != shB[0]) return ORC_ERR_SHAPE;
    int r = 0;
    for (int k = 0; k < rankA - 1; ++k) shD[r++] = shA[k];
    for (int k = 1; k < rankB; ++k) shD[r++] = shB[k];
    *rankD = r;
    return ORC_OK;
}

/* For output element `o` of the inner product (Eq. 2), build the index
 * vectors of A_{i..,p} and B_{p,j..} with the contracted position p left at
 * slot rankA-1 of ia and slot 0 of ib. */
static void inner_split(int64_t o, int rankA, const int64_t *shA, int rankB, const int64_t *shB,
                        int64_t *ia, int64_t *ib) {
    int64_t shD[MAXRANK], id[MAXRANK];
    int rD = 0;
    for (int k = 0; k < rankA - 1; ++k) shD[rD++] = shA[k];
    for (int k = 1; k < rankB; ++k) shD[rD++] = shB[k];
    psi_index(o, rD, shD, id);
    for (int k = 0; k < rankA - 1; ++k) ia[k] = id[k];
    for (int k = 1; k < rankB; ++k) ib[k] = id[rankA - 1 + k - 1];
    ia[rankA - 1] = 0;
    ib[0] = 0;
}

static int inner_check(int rankA, const int64_t *shA, int rankB, const int64_t *shB, int64_t *nD) {
    int rD;
    int64_t shD[MAXRANK];
    int st = oracle_inner_shape(rankA, shA, rankB, shB, &rD, shD);
    if (st) return st;
    *nD = tau(rD, shD);
    return ORC_OK;
}

/* ------------------------------------------------ error-free transformations */

/* TwoProduct via FMA: a*b = x + y exactly (Ogita, Rump & Oishi, "Accurate
 * sum and dot product", SIAM J. Sci. Comput. 26(6), 2005, Alg. 3.5). */
static void two_product(double a, double b, double *x, double *y) {
    *x = a * b;
    *y = fma(a, b, -*x);
}

/* TwoSum (Knuth): a+b = x + y exactly. */
static void two_sum(double a, double b, double *x, double *y) {
    *x = a + b;
    double z = *x - a;
    *y = (a - (*x - z)) + (b - z);
}

/* ------------------------------------------------------- inner, (+,x) */

/*
 * Eq. (2) with * = multiply and the sum over p: the matrix-multiply special
 * case generalised to any ranks.  Each output is the dot product of the
 * fibre A_{i..,:} with the fibre B_{:,j..}, evaluated by Dot2 (Ogita, Rump &
 * Oishi 2005, Alg. 5.3): as accurate as if computed in twice the working
 * precision and then rounded.  abs_out[k] = sum_p |A||B| (the normaliser of
 * the error measure |D - D_ref| / sum_p |A||B|).
 *
 * out_idx: flat output offsets to evaluate (NULL: all of them, in order).
 */
int oracle_inner_dot2(int rankA, const int64_t *shA, const double *A, int rankB, const int64_t *shB,
                      const double *B, int64_t n_out, const int64_t *out_idx, double *out, double *abs_out) {
    int64_t nD;
    int st = inner_check(rankA, shA, rankB, shB, &nD);
    if (st) return st;
    const int64_t P = shA[rankA - 1];
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nD) return ORC_ERR_INDEX;
        int64_t ia[MAXRANK], ib[MAXRANK];
        inner_split(o, rankA, shA, rankB, shB, ia, ib);
        double p_hi = 0.0, s = 0.0, a_sum = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            ia[rankA - 1] = p;
            ib[0] = p;
            double a = A[psi_offset(rankA, shA, ia)];
            double b = B[psi_offset(rankB, shB, ib)];
            double h, r, q;
            two_product(a, b, &h, &r);
            two_sum(p_hi, h, &p_hi, &q);
            s = s + (q + r);
            a_sum += fabs(a) * fabs(b);
        }
        out[k] = p_hi + s;
        if (abs_out) abs_out[k] = a_sum;
    }
    return ORC_OK;
}

/* ------------------------------------------- inner, FP32 semirings */

static float f32_combine(int op, float a, float b) {
    /* One FP32 operation, correctly rounded: computed exactly in binary64
     * (53 >= 2*24 + 2 makes the double rounding innocuous for + - * /;
     * Figueroa, "When is double rounding innocuous?", SIGNUM 1995). */
    double x = (double)a, y = (double)b;
    switch (op) {
    case OP_ADD: return (float)(x + y);
    case OP_SUB: return (float)(x - y);
    case OP_MUL: return (float)(x * y);
    case OP_DIV: return (float)(x / y);
    case OP_MIN: return fminf(a, b);
    case OP_MAX: return fmaxf(a, b);
    }
    return NAN;
}

static float f32_identity(int reduce) {
    /* The reduction starts from the identity of its operator (the appendix
     * accumulates into the result without showing how it was cleared). */
    switch (reduce) {
    case OP_MIN: return INFINITY;
    case OP_MAX: return -INFINITY;
    default: return 0.0f;
    }
}

/*
 * Eq. (2) generalised to D = reduce_p (A_{i..,p} combine B_{p,j..}) over
 * FP32 values, Sec. I letting the operation be any binary one: reduce min or
 * max, combine +, -, *, min or max ((min,+) shortest paths, (max,+) longest,
 * (max,*) most reliable, (max,min) widest / bottleneck, (min,max) minimax).
 * The fold starts at the reduction identity and runs in increasing p; min and
 * max make the result independent of that order.  NaN is treated as missing
 * (C99 fminf / fmaxf).
 */
int oracle_inner_f32(int reduce, int combine, int rankA, const int64_t *shA, const float *A, int rankB,
                     const int64_t *shB, const float *B, int64_t n_out, const int64_t *out_idx, float *out) {
    int64_t nD;
    int st = inner_check(rankA, shA, rankB, shB, &nD);
    if (st) return st;
    if (!(reduce == OP_MIN || reduce == OP_MAX)) return ORC_ERR_OP;
    if (!(combine == OP_ADD || combine == OP_MUL || combine == OP_SUB || combine == OP_MIN || combine == OP_MAX))
        return ORC_ERR_OP;
    const int64_t P = shA[rankA - 1];
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nD) return ORC_ERR_INDEX;
        int64_t ia[MAXRANK], ib[MAXRANK];
        inner_split(o, rankA, shA, rankB, shB, ia, ib);
        float acc = f32_identity(reduce);
        for (int64_t p = 0; p < P; ++p) {
            ia[rankA - 1] = p;
            ib[0] = p;
            float t = f32_combine(combine, A[psi_offset(rankA, shA, ia)], B[psi_offset(rankB, shB, ib)]);
            acc = f32_combine(reduce, acc, t);
        }
        out[k] = acc;
    }
    return ORC_OK;
}

/* Eq. (2) over 32-bit integers, (+,*) with two's-complement wraparound
 * (computed in uint32_t so overflow is defined). */
int oracle_inner_i32(int rankA, const int64_t *shA, const int32_t *A, int rankB, const int64_t *shB,
                     const int32_t *B, int64_t n_out, const int64_t *out_idx, int32_t *out) {
    int64_t nD;
    int st = inner_check(rankA, shA, rankB, shB, &nD);
    if (st) return st;
    const int64_t P = shA[rankA - 1];
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nD) return ORC_ERR_INDEX;
        int64_t ia[MAXRANK], ib[MAXRANK];
        inner_split(o, rankA, shA, rankB, shB, ia, ib);
        uint32_t acc = 0u;
        for (int64_t p = 0; p < P; ++p) {
            ia[rankA - 1] = p;
            ib[0] = p;
            uint32_t a = (uint32_t)A[psi_offset(rankA, shA, ia)];
            uint32_t b = (uint32_t)B[psi_offset(rankB, shB, ib)];
            acc = acc + a * b;
        }
        out[k] = (int32_t)acc;
    }
    return ORC_OK;
}

/* Eq. (2) over Booleans: D = OR_p (A_{i..,p} AND B_{p,j..}), one byte per
 * element (0 or 1) on input and output. */
int oracle_inner_bool(int rankA, const int64_t *shA, const uint8_t *A, int rankB, const int64_t *shB,
                      const uint8_t *B, int64_t n_out, const int64_t *out_idx, uint8_t *out) {
    int64_t nD;
    int st = inner_check(rankA, shA, rankB, shB, &nD);
    if (st) return st;
    const int64_t P = shA[rankA - 1];
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nD) return ORC_ERR_INDEX;
        int64_t ia[MAXRANK], ib[MAXRANK];
        inner_split(o, rankA, shA, rankB, shB, ia, ib);
        uint8_t acc = 0;
        for (int64_t p = 0; p < P; ++p) {
            ia[rankA - 1] = p;
            ib[0] = p;
            acc = acc | (A[psi_offset(rankA, shA, ia)] & B[psi_offset(rankB, shB, ib)]);
        }
        out[k] = acc ? 1 : 0;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ outer */

static uint16_t f32_to_bf16_rne(float f) {
    /* Round-to-nearest-even truncation of the low 16 bits of an FP32. */
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x40u); /* quiet NaN */
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static int outer_shape(int rankA, const int64_t *shA, int rankB, const int64_t *shB, int *rC, int64_t *shC) {
    /* Eq. (1): C_{ijkpqlm} = A_{ijkp} * B_{qlm}, so rho C = rho A ++ rho B. */
    if (rankA < 0 || rankB < 0 || rankA + rankB > MAXRANK) return ORC_ERR_RANK;
    int r = 0;
    for (int k = 0; k < rankA; ++k) shC[r++] = shA[k];
    for (int k = 0; k < rankB; ++k) shC[r++] = shB[k];
    *rC = r;
    return ORC_OK;
}

/*
 * Eq. (1) with a general binary operator (the paper names + - * / and
 * allows any binary operation; min and max are provided as well).
 * Operands are given exactly as doubles.  out_kind 0: the op in binary64;
 * 1: the op correctly rounded to FP32; 2: the FP32 result rounded again to
 * bfloat16 (RNE), stored as bit patterns.
 */
int oracle_outer_f(int op, int rankA, const int64_t *shA, const double *A, int rankB, const int64_t *shB,
                   const double *B, int out_kind, int64_t n_out, const int64_t *out_idx, void *out) {
    int rC;
    int64_t shC[MAXRANK], ic[MAXRANK];
    int st = outer_shape(rankA, shA, rankB, shB, &rC, shC);
    if (st) return st;
    if (op < OP_ADD || op > OP_MAX) return ORC_ERR_OP;
    const int64_t nC = tau(rC, shC);
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nC) return ORC_ERR_INDEX;
        psi_index(o, rC, shC, ic);
        double a = A[psi_offset(rankA, shA, ic)];
        double b = B[psi_offset(rankB, shB, ic + rankA)];
        double c;
        switch (op) {
        case OP_ADD: c = a + b; break;
        case OP_SUB: c = a - b; break;
        case OP_MUL: c = a * b; break;
        case OP_DIV: c = a / b; break;
        case OP_MIN: c = fmin(a, b); break;
        default: c = fmax(a, b); break;
        }
        if (out_kind == 0) ((double *)out)[k] = c;
        else if (out_kind == 1) ((float *)out)[k] = (float)c;
        else ((uint16_t *)out)[k] = f32_to_bf16_rne((float)c);
    }
    return ORC_OK;
}

/* Eq. (1) over 32-bit integers (+ - * with two's-complement wraparound). */
int oracle_outer_i32(int op, int rankA, const int64_t *shA, const int32_t *A, int rankB, const int64_t *shB,
                     const int32_t *B, int64_t n_out, const int64_t *out_idx, int32_t *out) {
    int rC;
    int64_t shC[MAXRANK], ic[MAXRANK];
    int st = outer_shape(rankA, shA, rankB, shB, &rC, shC);
    if (st) return st;
    if (op < OP_ADD || op > OP_MUL) return ORC_ERR_OP;
    const int64_t nC = tau(rC, shC);
    for (int64_t k = 0; k < n_out; ++k) {
        int64_t o = out_idx ? out_idx[k] : k;
        if (o < 0 || o >= nC) return ORC_ERR_INDEX;
        psi_index(o, rC, shC, ic);
        uint32_t a = (uint32_t)A[psi_offset(rankA, shA, ic)];
        uint32_t b = (uint32_t)B[psi_offset(rankB, shB, ic + rankA)];
        uint32_t c = op == OP_ADD ? a + b : op == OP_SUB ? a - b : a * b;
        out[k] = (int32_t)c;
    }
    return ORC_OK;
}

/* ------------------------------------------- appendix-order formulation */

/*
 * Row-at-a-time organisation of the inner product (Fig. 1; the appendix's
 * MoA routine is organised this way): the arrays are psi-flattened to an
 * M x K left operand, a K x N right operand and an M x N result (M = prod of
 * rho A without its last axis, K the contracted length, N = prod of rho B
 * without its first axis).  Result row i starts at the identity of the
 * reduce; then for every contraction position p, row p of the right operand
 * is combined with the single element A[i][p] and reduced into row i, one
 * element at a time along the row.  Result rows are shared among threads
 * round-robin (thread t owns rows t, t + T, t + 2T, ...), the thread
 * organisation of Sec. II.
 *
 * Plain recursive summation in the working type (no compensation).  This is
 * the second formulation the definition loops are cross-checked against, and
 * the loop the CPU baseline times.  kind: 0 f64 (+,*); 1 f32 with
 * (reduce, combine) (add,mul), or reduce min or max with combine add, sub,
 * mul, min or max (each step one correctly rounded FP32 operation, as in
 * the definition loop); 2 i32 (+,*) wrapping; 3 bool (or,and) bytes.
 */
int oracle_rowwise(int kind, int reduce, int combine, int rankA, const int64_t *shA, const void *A, int rankB,
                   const int64_t *shB, const void *B, void *D, int nthreads) {
    int64_t nD;
    int st = inner_check(rankA, shA, rankB, shB, &nD);
    if (st) return st;
    const int64_t M = tau(rankA - 1, shA);      /* result rows */
    const int64_t K = shA[rankA - 1];           /* contracted length */
    const int64_t N = tau(rankB - 1, shB + 1);  /* elements of a result row */
    if (nthreads < 1) nthreads = 1;
    if (kind == 1 && !((reduce == OP_ADD && combine == OP_MUL) ||
                       ((reduce == OP_MIN || reduce == OP_MAX) &&
                        (combine == OP_ADD || combine == OP_SUB || combine == OP_MUL || combine == OP_MIN ||
                         combine == OP_MAX))))
        return ORC_ERR_OP;
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < M; ++i) {
        if (kind == 0) {
            const double *a_row = (const double *)A + i * K;
            double *d_row = (double *)D + i * N;
            for (int64_t j = 0; j < N; ++j) d_row[j] = 0.0;
            for (int64_t p = 0; p < K; ++p) {
                const double alpha = a_row[p];
                const double *b_row = (const double *)B + p * N;
                for (int64_t j = 0; j < N; ++j) d_row[j] = d_row[j] + alpha * b_row[j];
            }
        } else if (kind == 1) {
            const float *a_row = (const float *)A + i * K;
            float *d_row = (float *)D + i * N;
            const float start = reduce == OP_ADD ? 0.0f : f32_identity(reduce);
            for (int64_t j = 0; j < N; ++j) d_row[j] = start;
            for (int64_t p = 0; p < K; ++p) {
                const float alpha = a_row[p];
                const float *b_row = (const float *)B + p * N;
                for (int64_t j = 0; j < N; ++j) d_row[j] = f32_combine(reduce, d_row[j], f32_combine(combine, alpha, b_row[j]));
            }
        } else if (kind == 2) {
            const int32_t *a_row = (const int32_t *)A + i * K;
            uint32_t *d_row = (uint32_t *)D + i * N;
            for (int64_t j = 0; j < N; ++j) d_row[j] = 0u;
            for (int64_t p = 0; p < K; ++p) {
                const uint32_t alpha = (uint32_t)a_row[p];
                const int32_t *b_row = (const int32_t *)B + p * N;
                for (int64_t j = 0; j < N; ++j) d_row[j] = d_row[j] + alpha * (uint32_t)b_row[j];
            }
        } else {
            const uint8_t *a_row = (const uint8_t *)A + i * K;
            uint8_t *d_row = (uint8_t *)D + i * N;
            for (int64_t j = 0; j < N; ++j) d_row[j] = 0;
            for (int64_t p = 0; p < K; ++p) {
                const uint8_t alpha = a_row[p];
                const uint8_t *b_row = (const uint8_t *)B + p * N;
                for (int64_t j = 0; j < N; ++j) d_row[j] = d_row[j] | (alpha & b_row[j]);
            }
        }
    }
    return ORC_OK;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
