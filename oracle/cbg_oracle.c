/*
 * cbg_oracle.c -- plain CPU FP64 oracle for compressed-basis GMRES.
 *
 * TEST INFRASTRUCTURE ONLY (see cbg_oracle.h for what it follows and the readings it
 * takes).  No fused operations: the build uses -ffp-contract=off so that every product
 * and sum is rounded separately, on x86 and on aarch64 alike.
 *
 * Parallel loops (OpenMP, when the build enables it) only split work whose result does
 * not depend on the split: rows of a sparse product, elements of a vector update, and
 * the fixed blocks of an inner product (reading R19: every inner product adds its terms
 * in index order within blocks of OR_DOT_BLOCK terms, then the block sums in block
 * order).  One thread and all threads give bitwise the same results.
 */
#include "cbg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* loops shorter than this stay on one thread (the parallel region would cost more) */
#define OR_PAR_MIN 32768

void or_set_threads(int t)
{
#ifdef _OPENMP
    omp_set_num_threads(t < 1 ? 1 : t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ===================================================================================
 * Scalar codec, written from the format definitions.
 *
 * A binary floating-point format with p significand bits (hidden bit included),
 * minimum normal exponent emin and maximum exponent emax represents the values
 *   k * 2^q   with integer k, |k| < 2^p, and q >= emin - (p - 1).
 * Round-to-nearest-even of a real x: pick the quantum q = max(E, emin) - (p - 1) where
 * 2^E <= |x| < 2^(E+1), round |x| / 2^q to the nearest integer (ties to the even one),
 * and scale back.  All steps below are exact in FP64 for the formats used here.
 * =================================================================================== */
static double round_to_format(double x, int p, int emin)
{
    if (x == 0.0 || !isfinite(x)) return x;
    double ax = fabs(x);
    int e2;
    (void)frexp(ax, &e2);          /* ax = f * 2^e2, f in [0.5, 1) */
    int E = e2 - 1;                /* 2^E <= ax < 2^(E+1)          */
    int q = (E < emin ? emin : E) - (p - 1);
    double s = ldexp(ax, -q);      /* exact: only the exponent changes */
    double k = floor(s);
    double rem = s - k;            /* exact: s < 2^(p+1) * 2 */
    if (rem > 0.5 || (rem == 0.5 && fmod(k, 2.0) != 0.0)) k += 1.0;
    return copysign(ldexp(k, q), x);
}

/* Exponent and mantissa fields (sign excluded) of an exactly representable value r of
 * a format with mbits = p - 1 stored mantissa bits and exponent bias `bias`. */
static uint32_t pack_format(double r, int mbits, int bias, int emin)
{
    double a = fabs(r);
    uint32_t expf, man;
    if (a == 0.0) {
        expf = 0; man = 0;
    } else {
        int e2;
        (void)frexp(a, &e2);
        int E = e2 - 1;
        if (E < emin) {                       /* subnormal: a = man * 2^(emin - mbits) */
            expf = 0;
            man = (uint32_t)ldexp(a, mbits - emin);
        } else {                              /* normal: a = (2^mbits + man) 2^(E - mbits) */
            expf = (uint32_t)(E + bias);
            man = (uint32_t)(ldexp(a, mbits - E) - ldexp(1.0, mbits));
        }
    }
    return (expf << mbits) | man;
}

static double unpack_format(uint32_t expf, uint32_t man, int mbits, int bias, int emin)
{
    if (expf == 0) return ldexp((double)man, emin - mbits);
    return ldexp((double)((1u << mbits) + man), (int)expf - bias - mbits);
}

/* ---- IEEE binary16: p = 11, emin = -14, emax = 15, bias 15 ------------------------ */
uint16_t or_f64_to_f16(double x)
{
    uint16_t sign = signbit(x) ? 0x8000u : 0u;
    if (isnan(x)) return (uint16_t)(sign | 0x7E00u);
    double r = round_to_format(x, 11, -14);
    if (fabs(r) > 65504.0) return (uint16_t)(sign | 0x7C00u);   /* overflow -> inf */
    uint32_t bits = pack_format(r, 10, 15, -14);
    return (uint16_t)(sign | bits);
}

double or_f16_to_f64(uint16_t h)
{
    uint32_t expf = (h >> 10) & 0x1Fu, man = h & 0x3FFu;
    double s = (h & 0x8000u) ? -1.0 : 1.0;
    if (expf == 0x1Fu) return man ? NAN : s * INFINITY;
    return s * unpack_format(expf, man, 10, 15, -14);
}

/* ---- bfloat16: p = 8, emin = -126, emax = 127, bias 127 --------------------------- */
uint16_t or_f32_to_bf16(float xf)
{
    double x = (double)xf;
    uint16_t sign = signbit(x) ? 0x8000u : 0u;
    if (isnan(x)) return (uint16_t)(sign | 0x7FC0u);
    if (isinf(x)) return (uint16_t)(sign | 0x7F80u);
    double r = round_to_format(x, 8, -126);
    if (fabs(r) > 0x1.FEp127) return (uint16_t)(sign | 0x7F80u);
    uint32_t bits = pack_format(r, 7, 127, -126);
    return (uint16_t)(sign | bits);
}

double or_bf16_to_f64(uint16_t b)
{
    uint32_t expf = (b >> 7) & 0xFFu, man = b & 0x7Fu;
    double s = (b & 0x8000u) ? -1.0 : 1.0;
    if (expf == 0xFFu) return man ? NAN : s * INFINITY;
    return s * unpack_format(expf, man, 7, 127, -126);
}

/* ---- OCP FP8 E4M3 ("fn": no infinities): p = 4, emin = -6, bias 7, max 448 ---------
 * S.1111.111 is NaN; every other pattern is finite.  Saturating conversion: results
 * beyond 448 in magnitude (including infinities) become +-448. */
uint8_t or_f32_to_e4m3(float xf)
{
    double x = (double)xf;
    uint8_t sign = signbit(x) ? 0x80u : 0u;
    if (isnan(x)) return 0x7Fu;
    double r = isinf(x) ? copysign(448.0, x) : round_to_format(x, 4, -6);
    if (fabs(r) > 448.0) r = copysign(448.0, x);
    uint32_t bits = pack_format(r, 3, 7, -6);
    return (uint8_t)(sign | bits);
}

double or_e4m3_to_f64(uint8_t c)
{
    uint32_t expf = (c >> 3) & 0xFu, man = c & 0x7u;
    double s = (c & 0x80u) ? -1.0 : 1.0;
    if (expf == 0xFu && man == 0x7u) return NAN;
    return s * unpack_format(expf, man, 3, 7, -6);
}

int or_format_bytes(int fmt)
{
    switch (fmt) {
    case OR_F64: return 8;
    case OR_F32: case OR_I32: return 4;
    case OR_F16: case OR_BF16: case OR_I16: return 2;
    case OR_E4M3: return 1;
    default: return 0;
    }
}

/* ===================================================================================
 * Vector codec (Section 4.2 memory accessor).
 * =================================================================================== */
static double int_max(int fmt) { return fmt == OR_I32 ? 2147483647.0 : 32767.0; }

/* smallest integer e with vmax <= fmax * 2^e (reading R5) */
static int pow2_scale_exponent(double vmax, double fmax)
{
    int e2;
    (void)frexp(vmax, &e2);
    int e = e2 - 12;                       /* well below the answer for both formats */
    while (vmax > ldexp(fmax, e)) e += 1;
    if (e < -126) e = -126;                /* keep the scale a normal FP32 number */
    return e;
}

int or_encode(int fmt, int64_t n, const double* v, double vmax, void* codes, double* scale)
{
    if (n < 0 || (n > 0 && (!v || !codes)) || !scale) return OR_ERR_ARG;
    if (!(vmax > 0.0)) vmax = 1.0;          /* all-zero vector: any scale encodes it */
    switch (fmt) {
    case OR_F64: {
        double* c = (double*)codes;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) c[i] = v[i];
        *scale = 1.0;
        return OR_OK;
    }
    case OR_F32: {
        float* c = (float*)codes;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) c[i] = (float)v[i];
        *scale = 1.0;
        return OR_OK;
    }
    case OR_F16: {
        uint16_t* c = (uint16_t*)codes;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) c[i] = or_f64_to_f16(v[i]);
        *scale = 1.0;
        return OR_OK;
    }
    case OR_I32:
    case OR_I16: {
        double mx = int_max(fmt);
        double sigma = vmax / mx;           /* sigma_j = (||w||_inf/||w||_2) / max_int */
        double inv = 1.0 / sigma;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) {
            double q = rint(v[i] * inv);
            if (q > mx) q = mx;
            if (q < -mx) q = -mx;
            if (fmt == OR_I32) ((int32_t*)codes)[i] = (int32_t)q;
            else ((int16_t*)codes)[i] = (int16_t)q;
        }
        *scale = sigma;
        return OR_OK;
    }
    case OR_BF16:
    case OR_E4M3: {
        int e = pow2_scale_exponent(vmax, fmt == OR_BF16 ? 1.0 : 448.0);
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) {
            float f = (float)ldexp(v[i], -e);
            if (fmt == OR_BF16) ((uint16_t*)codes)[i] = or_f32_to_bf16(f);
            else ((uint8_t*)codes)[i] = or_f32_to_e4m3(f);
        }
        *scale = ldexp(1.0, e);
        return OR_OK;
    }
    default:
        return OR_ERR_ARG;
    }
}

int or_decode(int fmt, int64_t n, const void* codes, double scale, double* out)
{
    if (n < 0 || (n > 0 && (!codes || !out))) return OR_ERR_ARG;
    if (or_format_bytes(fmt) == 0) return OR_ERR_ARG;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; i++) {
        switch (fmt) {
        case OR_F64: out[i] = ((const double*)codes)[i]; break;
        case OR_F32: out[i] = (double)((const float*)codes)[i]; break;
        case OR_F16: out[i] = or_f16_to_f64(((const uint16_t*)codes)[i]); break;
        case OR_I32: out[i] = (double)((const int32_t*)codes)[i] * scale; break;
        case OR_I16: out[i] = (double)((const int16_t*)codes)[i] * scale; break;
        case OR_BF16: out[i] = or_bf16_to_f64(((const uint16_t*)codes)[i]) * scale; break;
        case OR_E4M3: out[i] = or_e4m3_to_f64(((const uint8_t*)codes)[i]) * scale; break;
        default: break;
        }
    }
    return OR_OK;
}

/* ===================================================================================
 * Building blocks.
 * =================================================================================== */
void or_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             const double* x, double* y)
{
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * x[col[p]];
        y[i] = s;
    }
}

/* sum of a_i b_i (reading R19): terms in index order within each block of OR_DOT_BLOCK,
 * then the block sums in block order */
double or_dot(int64_t n, const double* a, const double* b)
{
    if (n <= 0) return 0.0;
    const int64_t nb = (n + OR_DOT_BLOCK - 1) / OR_DOT_BLOCK;
    double stack_part[64];
    double* part = nb <= 64 ? stack_part : (double*)malloc((size_t)nb * sizeof(double));
    if (!part) return NAN;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t k = 0; k < nb; k++) {
        const int64_t i1 = (k + 1) * OR_DOT_BLOCK < n ? (k + 1) * OR_DOT_BLOCK : n;
        double s = 0.0;
        for (int64_t i = k * OR_DOT_BLOCK; i < i1; i++) s += a[i] * b[i];
        part[k] = s;
    }
    double s = 0.0;
    for (int64_t k = 0; k < nb; k++) s += part[k];
    if (part != stack_part) free(part);
    return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(or_dot(n, a, a)); }

static double nrminf(int64_t n, const double* a)
{
    double m = 0.0;   /* the maximum does not depend on the order */
#pragma omp parallel for schedule(static) reduction(max : m) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; i++) if (fabs(a[i]) > m) m = fabs(a[i]);
    return m;
}

static int all_finite(int64_t n, const double* a)
{
    int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; i++) ok = ok && isfinite(a[i]);
    return ok;
}

typedef struct {
    int64_t n;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    int precond;
    const double* dinv_src;   /* diagonal of A (Jacobi) */
    const double* pvals;      /* SPAI values          */
    const double* binv;       /* block-Jacobi: inverse of diagonal block b, row-major 4x4 at 16 b */
} problem;

/* Inverse of the diagonal blocks of A (rows and columns 4b .. 4b+3, the last block
 * possibly smaller) by Gauss-Jordan elimination on [D | I] with partial pivoting (the
 * largest |entry| of the column at or below the diagonal).  Returns 0, or -1 if a block
 * is singular. */
static int block_jacobi_inverse(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                                double* binv)
{
    for (int64_t r0 = 0; r0 < n; r0 += 4) {
        const int kb = (int)(n - r0 < 4 ? n - r0 : 4);
        double aug[4][8];
        for (int i = 0; i < kb; i++) {
            for (int c = 0; c < 2 * kb; c++) aug[i][c] = (c == kb + i) ? 1.0 : 0.0;
            for (int32_t p = rowptr[r0 + i]; p < rowptr[r0 + i + 1]; p++) {
                const int64_t c = col[p] - r0;
                if (c >= 0 && c < kb) aug[i][c] = val[p];
            }
        }
        for (int k = 0; k < kb; k++) {
            int piv = k;
            for (int i = k + 1; i < kb; i++)
                if (fabs(aug[i][k]) > fabs(aug[piv][k])) piv = i;
            if (aug[piv][k] == 0.0) return -1;
            for (int c = 0; c < 2 * kb; c++) {
                const double t = aug[k][c];
                aug[k][c] = aug[piv][c];
                aug[piv][c] = t;
            }
            const double d = aug[k][k];
            for (int c = 0; c < 2 * kb; c++) aug[k][c] = aug[k][c] / d;
            for (int i = 0; i < kb; i++) {
                if (i == k) continue;
                const double f = aug[i][k];
                for (int c = 0; c < 2 * kb; c++) aug[i][c] = aug[i][c] - f * aug[k][c];
            }
        }
        double* B = binv + 16 * (r0 / 4);
        for (int i = 0; i < kb; i++)
            for (int c = 0; c < kb; c++) B[4 * i + c] = aug[i][kb + c];
    }
    return 0;
}

/* z = M^{-1} v  (Fig. 1: the Arnoldi SpMV and the solution update; right preconditioning) */
static void apply_precond(const problem* P, const double* v, double* z)
{
    int64_t n = P->n;
    if (P->precond == OR_PC_JACOBI) {
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) z[i] = v[i] / P->dinv_src[i];
    } else if (P->precond == OR_PC_SPAI) {
        or_spmv(n, P->rowptr, P->col, P->pvals, v, z);
    } else if (P->precond == OR_PC_BJ4) {
        for (int64_t r0 = 0; r0 < n; r0 += 4) {
            const int kb = (int)(n - r0 < 4 ? n - r0 : 4);
            const double* B = P->binv + 16 * (r0 / 4);
            for (int i = 0; i < kb; i++) {
                double s = 0.0;
                for (int c = 0; c < kb; c++) s += B[4 * i + c] * v[r0 + c];
                z[r0 + i] = s;
            }
        }
    } else {
        memcpy(z, v, (size_t)n * sizeof(double));
    }
}

/* Normalise w by the FP64 reciprocal of h (reading R3), store it in the basis format,
 * and put the decoded vector in vt (the oracle computes with what the GPU stores). */
static int compress_column(int fmt, int64_t n, const double* w, double h, void* codes,
                           double* vt, double* tmp)
{
    double inv = 1.0 / h;
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; i++) tmp[i] = w[i] * inv;
    double vmax = nrminf(n, tmp);
    double scale;
    int rc = or_encode(fmt, n, tmp, vmax, codes, &scale);
    if (rc) return rc;
    return or_decode(fmt, n, codes, scale, vt);
}

/* Adaptive basis format (reading R15; the paper fixes one format per solve): the next
 * format up the ladder e4m3 -> bf16 -> f32 -> f64, f16 -> f32, i16 -> i32 -> f64, or -1. */
/* One Gram-Schmidt pass of w against the columns 0..ncols-1 of V (n x ncols,
 * column-major), the coefficients into c.  CGS (Fig. 1): every coefficient from the same
 * w, then w -= V c.  MGS (the variant Section 2 mentions): column by column, the
 * coefficient from the current w, which that column then reduces at once. */
void or_gram_schmidt_pass(int64_t n, const double* V, int64_t ncols, int ortho, double* w, double* c)
{
    const int64_t j = ncols - 1;
    if (ortho == OR_ORTHO_MGS) {
        for (int64_t i = 0; i <= j; i++) {
            const double* vi = V + (size_t)i * (size_t)n;
            c[i] = or_dot(n, vi, w);
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t t = 0; t < n; t++) w[t] -= vi[t] * c[i];
        }
        return;
    }
    for (int64_t i = 0; i <= j; i++) c[i] = or_dot(n, V + (size_t)i * (size_t)n, w);
    /* w -= V c: every element subtracts its terms in column order 0..j */
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t t = 0; t < n; t++) {
        double wt = w[t];
        for (int64_t i = 0; i <= j; i++) wt -= V[(size_t)i * (size_t)n + (size_t)t] * c[i];
        w[t] = wt;
    }
}

static int wider_format(int f)
{
    if (f == OR_E4M3) return OR_BF16;
    if (f == OR_BF16 || f == OR_F16) return OR_F32;
    if (f == OR_I16) return OR_I32;
    if (f == OR_F32 || f == OR_I32) return OR_F64;
    return -1;
}

/* ===================================================================================
 * GMRES(m), Fig. 1, with the explicit-residual recheck of Section 5.2.
 * =================================================================================== */
int or_gmres(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             const double* b, double* x, or_gmres_args* a)
{
    if (!a) return OR_ERR_ARG;
    a->iters = a->cycles = a->reorths = a->k1 = a->nhist = a->ntres = 0;
    a->true_relres = a->est_relres = 0.0;
    a->status = OR_ERR_ARG;
    if (n <= 0 || !rowptr || !col || !val || !b || !x || a->m < 1 || a->maxit < 0 ||
        or_format_bytes(a->fmt) == 0 || !(a->tol >= 0.0))
        return a->status;
    if (a->precond == OR_PC_SPAI && !a->pvals) return a->status;
    int64_t nnz = rowptr[n];
    const int m = a->m;

    if (!all_finite(n, b) || !all_finite(nnz, val) || !all_finite(n, x) ||
        (a->precond == OR_PC_SPAI && !all_finite(nnz, a->pvals))) {
        a->status = OR_ERR_NONFINITE;
        return a->status;
    }

    problem P = {n, rowptr, col, val, a->precond, NULL, a->pvals, NULL};
    double* diag = NULL;
    double* binv = NULL;
    if (a->precond == OR_PC_BJ4) {
        binv = (double*)calloc((size_t)(16 * ((n + 3) / 4)), sizeof(double));
        if (!binv || block_jacobi_inverse(n, rowptr, col, val, binv)) { free(binv); return a->status; }
        P.binv = binv;
    }
    if (a->precond == OR_PC_JACOBI) {
        diag = (double*)calloc((size_t)n, sizeof(double));
        for (int64_t i = 0; i < n; i++)
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++)
                if (col[p] == i) diag[i] = val[p];
        for (int64_t i = 0; i < n; i++)
            if (diag[i] == 0.0) { free(diag); free(binv); return a->status; }
        P.dinv_src = diag;
    }

    const double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {                                  /* reading R8 */
        for (int64_t i = 0; i < n; i++) x[i] = 0.0;
        a->status = OR_OK;
        free(diag);
        free(binv);
        return a->status;
    }
    const double target = a->tol * bnorm;

    /* basis: decoded columns (what every use of V_j sees) and one code buffer */
    int64_t kcap_all = a->maxit < m ? a->maxit : m;
    int64_t ncols = kcap_all + 1;
    double* V = (double*)malloc((size_t)n * (size_t)ncols * sizeof(double));
    void* codes = malloc((size_t)n * 8);
    double* r = (double*)malloc((size_t)n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* z = (double*)malloc((size_t)n * sizeof(double));
    double* tmp = (double*)malloc((size_t)n * sizeof(double));
    double* H = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* raw    */
    double* R = (double*)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* rotated */
    double* cs = (double*)calloc((size_t)m, sizeof(double));
    double* sn = (double*)calloc((size_t)m, sizeof(double));
    double* g = (double*)calloc((size_t)m + 1, sizeof(double));
    double* h = (double*)calloc((size_t)m + 1, sizeof(double));
    double* u = (double*)calloc((size_t)m + 1, sizeof(double));
    double* y = (double*)calloc((size_t)m, sizeof(double));
    if (!V || !codes || !r || !w || !z || !tmp || !H || !R || !cs || !sn || !g || !h || !u || !y) {
        a->status = OR_ERR_ARG;
        goto done;
    }

    int fmt = a->fmt;            /* basis format of the current cycle (adapt moves it up) */
    double last_est = 0.0;       /* recurrence residual the previous cycle ended with   */
    a->promotions = 0;
    for (;;) {
        /* Fig. 1, cycle start: r0 = b - A x0, beta = ||r0|| */
        or_spmv(n, rowptr, col, val, x, r);
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];
        double beta = nrm2(n, r);
        if (!isfinite(beta)) { a->status = OR_ERR_NONFINITE; break; }
        a->true_relres = beta / bnorm;
        if (a->tres && a->ntres < a->tres_cap) a->tres[a->ntres++] = beta / bnorm;
        if (beta <= target) { a->status = OR_OK; break; }
        if (a->iters >= a->maxit) { a->status = OR_NOT_CONVERGED; break; }
        /* adapt: the explicit residual exceeds adapt_gap times what the last cycle's
         * recurrence promised -> the compressed basis limits the solve: widen it */
        if (a->adapt && a->cycles > 0 && beta > a->adapt_gap * last_est) {
            const int wf = wider_format(fmt);
            if (wf >= 0) {
                fmt = wf;
                a->promotions++;
            }
        }
        a->cycles++;
        int64_t kcap = a->maxit - a->iters;
        if (kcap > m) kcap = m;

        /* v = r0 / beta, stored compressed: V_1 = [v] */
        if (compress_column(fmt, n, r, beta, codes, V, tmp)) { a->status = OR_ERR_ARG; break; }
        memset(R, 0, (size_t)(m + 1) * (size_t)m * sizeof(double));
        memset(H, 0, (size_t)(m + 1) * (size_t)m * sizeof(double));
        memset(g, 0, ((size_t)m + 1) * sizeof(double));
        g[0] = beta;

        int64_t k = 0;           /* columns of H completed in this cycle */
        int64_t nv = 1;          /* basis vectors stored in this cycle    */
        int nonfinite = 0;
        for (int64_t j = 0; j < kcap; j++) {
            const double* vj = V + (size_t)j * (size_t)n;
            /* w = A (M^{-1} v) */
            apply_precond(&P, vj, z);
            or_spmv(n, rowptr, col, val, z, w);
            /* omega = ||w|| */
            double omega = nrm2(n, w);
            /* Gram-Schmidt: h_{1:j,j} = V_j^T w, w = w - V_j h (CGS; or MGS) */
            or_gram_schmidt_pass(n, V, j + 1, a->ortho, w, h);
            /* h_{j+1,j} = ||w|| */
            double hn = nrm2(n, w);
            /* re-orthogonalise (always, or when h_{j+1,j} < eta omega) */
            int do_re = a->reorth == OR_REORTH_ALWAYS ||
                        (a->reorth == OR_REORTH_CONDITIONAL && hn < a->eta * omega);
            if (do_re) {
                or_gram_schmidt_pass(n, V, j + 1, a->ortho, w, u);
                for (int64_t i = 0; i <= j; i++) h[i] += u[i];
                hn = nrm2(n, w);
                a->reorths++;
            }
            if (!isfinite(hn) || !isfinite(omega)) { nonfinite = 1; break; }
            /* column j of the (m+1) x m Hessenberg (Fig. 1) */
            for (int64_t i = 0; i <= j; i++) H[i + j * (m + 1)] = h[i];
            H[j + 1 + j * (m + 1)] = hn;
            a->iters++;

            /* Section 2: QR of the Hessenberg updated by one Givens rotation per column */
            double* Rc = R + j * (m + 1);
            for (int64_t i = 0; i <= j + 1; i++) Rc[i] = H[i + j * (m + 1)];
            for (int64_t i = 0; i < j; i++) {
                double t0 = cs[i] * Rc[i] + sn[i] * Rc[i + 1];
                double t1 = -sn[i] * Rc[i] + cs[i] * Rc[i + 1];
                Rc[i] = t0;
                Rc[i + 1] = t1;
            }
            double rr = hypot(Rc[j], Rc[j + 1]);
            if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = Rc[j] / rr; sn[j] = Rc[j + 1] / rr; }
            Rc[j] = rr;
            Rc[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            double est = fabs(g[j + 1]);
            last_est = est;
            a->est_relres = est / bnorm;
            if (a->hist && a->nhist < a->hist_cap) a->hist[a->nhist++] = est / bnorm;
            k = j + 1;

            /* breakdown (reading R2) or the printed clause */
            int stop = !(hn > a->eps_bd * omega);
            if (a->literal_fig1) stop = (hn == 0.0) || (hn < a->eta * omega);
            if (stop) break;
            /* recurrence residual signals convergence (Section 5.2) */
            if (est <= target) break;
            /* v = w / h_{j+1,j}, V_{j+1} = [V_j, v] (stored compressed) */
            if (compress_column(fmt, n, w, hn, codes, V + (size_t)(j + 1) * (size_t)n, tmp)) {
                nonfinite = 1;
                break;
            }
            nv = j + 2;
        }
        if (nonfinite) { a->status = OR_ERR_NONFINITE; break; }
        if (a->cycles == 1) {
            a->k1 = k;
            if (a->H1) memcpy(a->H1, H, (size_t)(m + 1) * (size_t)m * sizeof(double));
            if (a->V1) memcpy(a->V1, V, (size_t)n * (size_t)nv * sizeof(double));
        }
        /* y = argmin ||beta e1 - H y|| by back substitution on R */
        for (int64_t i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int64_t c = i + 1; c < k; c++) s -= R[i + c * (m + 1)] * y[c];
            y[i] = s / R[i + i * (m + 1)];
        }
        /* x = x0 + M^{-1} (V_k y); every element adds its terms in column order */
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t t = 0; t < n; t++) {
            double s = 0.0;
            for (int64_t c = 0; c < k; c++) s += V[(size_t)c * (size_t)n + (size_t)t] * y[c];
            tmp[t] = s;
        }
        apply_precond(&P, tmp, z);
#pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t t = 0; t < n; t++) x[t] += z[t];
        if (!all_finite(n, x)) { a->status = OR_ERR_NONFINITE; break; }
        /* restart (the explicit residual decides) */
    }
done:
    a->fmt_final = fmt;
    free(V); free(codes); free(r); free(w); free(z); free(tmp); free(H); free(R);
    free(cs); free(sn); free(g); free(h); free(u); free(y); free(diag); free(binv);
    return a->status;
}

/* ===================================================================================
 * Learned SPAI preconditioner: per-row MLP 7 -> 64 -> 64 -> 7 with ReLU, in FP64.
 *   a1 = relu(W1 f + b1), a2 = relu(W2 a1 + b2), out = W3 a2 + b3
 * W1: 64 x 7, W2: 64 x 64, W3: 7 x 64, row-major (out x in).
 * =================================================================================== */
#define MLP_IN 7
#define MLP_H 64
#define MLP_OUT 7

static void mlp_row(const double* f, const double* W1, const double* b1, const double* W2,
                    const double* b2, const double* W3, const double* b3, double* a1,
                    double* a2, double* out)
{
    for (int o = 0; o < MLP_H; o++) {
        double s = b1[o];
        for (int i = 0; i < MLP_IN; i++) s += W1[o * MLP_IN + i] * f[i];
        a1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < MLP_H; o++) {
        double s = b2[o];
        for (int i = 0; i < MLP_H; i++) s += W2[o * MLP_H + i] * a1[i];
        a2[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < MLP_OUT; o++) {
        double s = b3[o];
        for (int i = 0; i < MLP_H; i++) s += W3[o * MLP_H + i] * a2[i];
        out[o] = s;
    }
}

int or_mlp_forward(int64_t rows, const double* feat, const double* W1, const double* b1,
                   const double* W2, const double* b2, const double* W3, const double* b3,
                   double* out, double* act1, double* act2)
{
    double a1[MLP_H], a2[MLP_H];
    for (int64_t r = 0; r < rows; r++) {
        mlp_row(feat + r * MLP_IN, W1, b1, W2, b2, W3, b3, a1, a2, out + r * MLP_OUT);
        if (act1) memcpy(act1 + r * MLP_H, a1, sizeof a1);
        if (act2) memcpy(act2 + r * MLP_H, a2, sizeof a2);
    }
    return OR_OK;
}

int or_mlp_backward(int64_t rows, const double* feat, const double* W1, const double* b1,
                    const double* W2, const double* b2, const double* W3, const double* b3,
                    const double* gout, double* gW1, double* gb1, double* gW2, double* gb2,
                    double* gW3, double* gb3)
{
    memset(gW1, 0, sizeof(double) * MLP_H * MLP_IN); memset(gb1, 0, sizeof(double) * MLP_H);
    memset(gW2, 0, sizeof(double) * MLP_H * MLP_H);  memset(gb2, 0, sizeof(double) * MLP_H);
    memset(gW3, 0, sizeof(double) * MLP_OUT * MLP_H); memset(gb3, 0, sizeof(double) * MLP_OUT);
    double a1[MLP_H], a2[MLP_H], out[MLP_OUT], d2[MLP_H], d1[MLP_H];
    for (int64_t r = 0; r < rows; r++) {
        const double* f = feat + r * MLP_IN;
        const double* go = gout + r * MLP_OUT;
        mlp_row(f, W1, b1, W2, b2, W3, b3, a1, a2, out);
        for (int o = 0; o < MLP_OUT; o++) {
            gb3[o] += go[o];
            for (int i = 0; i < MLP_H; i++) gW3[o * MLP_H + i] += go[o] * a2[i];
        }
        for (int i = 0; i < MLP_H; i++) {
            double s = 0.0;
            for (int o = 0; o < MLP_OUT; o++) s += W3[o * MLP_H + i] * go[o];
            d2[i] = a2[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < MLP_H; o++) {
            gb2[o] += d2[o];
            for (int i = 0; i < MLP_H; i++) gW2[o * MLP_H + i] += d2[o] * a1[i];
        }
        for (int i = 0; i < MLP_H; i++) {
            double s = 0.0;
            for (int o = 0; o < MLP_H; o++) s += W2[o * MLP_H + i] * d2[o];
            d1[i] = a1[i] > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < MLP_H; o++) {
            gb1[o] += d1[o];
            for (int i = 0; i < MLP_IN; i++) gW1[o * MLP_IN + i] += d1[o] * f[i];
        }
    }
    return OR_OK;
}

/* ---- element-wise helpers used by the codec pins (no scale) ------------------------ */
void or_vec_f64_to_f16(int64_t n, const double* x, uint16_t* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_f64_to_f16(x[i]); }
void or_vec_f16_to_f64(int64_t n, const uint16_t* c, double* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_f16_to_f64(c[i]); }
void or_vec_f32_to_bf16(int64_t n, const float* x, uint16_t* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_f32_to_bf16(x[i]); }
void or_vec_bf16_to_f64(int64_t n, const uint16_t* c, double* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_bf16_to_f64(c[i]); }
void or_vec_f32_to_e4m3(int64_t n, const float* x, uint8_t* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_f32_to_e4m3(x[i]); }
void or_vec_e4m3_to_f64(int64_t n, const uint8_t* c, double* out)
{ for (int64_t i = 0; i < n; i++) out[i] = or_e4m3_to_f64(c[i]); }

/* ===================================================================================
 * Learned SPAI statistics (quadratic loss in the per-row SPAI values).
 * =================================================================================== */
int or_spai_slots(int64_t n, const int32_t* rowptr, const int32_t* col, int64_t sx, int64_t sxy,
                  int8_t* slot)
{
    const int64_t off[7] = {-sxy, -sx, -1, 0, 1, sx, sxy};
    for (int64_t i = 0; i < n; i++)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int64_t dlt = (int64_t)col[p] - i;
            int k = -1;
            for (int t = 0; t < 7; t++) if (off[t] == dlt) k = t;
            if (k < 0) return OR_ERR_ARG;
            slot[p] = (int8_t)k;
        }
    return OR_OK;
}

int or_spai_accumulate(int64_t n, const int32_t* rowptr, const int32_t* col, const int8_t* slot,
                       const double* r, const double* e, double wgt, double* G, double* c, double* d)
{
    for (int64_t i = 0; i < n; i++) {
        double rv[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) rv[slot[p]] = r[col[p]];
        for (int k = 0; k < 7; k++) {
            for (int l = 0; l < 7; l++) G[i * 49 + k * 7 + l] += wgt * rv[k] * rv[l];
            c[i * 7 + k] += wgt * e[i] * rv[k];
        }
        d[i] += wgt * e[i] * e[i];
    }
    return OR_OK;
}

double or_spai_loss(int64_t n, const int32_t* rowptr, const int8_t* slot, const double* out,
                    const double* diag, const double* G, const double* c, const double* d,
                    double npairs, double* gout)
{
    double loss = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double pv[7] = {0, 0, 0, 0, 0, 0, 0};
        int has[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; p++) has[slot[p]] = 1;
        for (int k = 0; k < 7; k++) pv[k] = has[k] ? out[i * 7 + k] / diag[i] : 0.0;
        double li = d[i];
        for (int k = 0; k < 7; k++) {
            double gp = 0.0;
            for (int l = 0; l < 7; l++) gp += G[i * 49 + k * 7 + l] * pv[l];
            li += pv[k] * gp - 2.0 * pv[k] * c[i * 7 + k];
            if (gout) gout[i * 7 + k] = has[k] ? 2.0 * (gp - c[i * 7 + k]) / diag[i] / npairs : 0.0;
        }
        loss += li;
    }
    return loss / npairs;
}
