/*
 * cbg_oracle.h -- plain CPU FP64 oracle for compressed-basis GMRES (CB-GMRES).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a deliberately slow, sequential, obviously
 * correct restatement of the method of Aliaga, Anzt, Gruetzmacher, Quintana-Orti and
 * Tomas, "Compressed Basis GMRES on High Performance GPUs" (arXiv 2009.12101).  Only
 * the tests, the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library; the two only see
 * the same seeded inputs.
 *
 * What it follows:
 *   - Fig. 1 (restarted, right-preconditioned GMRES(m) with classical Gram-Schmidt and
 *     optional re-orthogonalisation), step by step;
 *   - Section 2 (stopping test ||b - A x||_2 <= tau ||b||_2, QR/Givens update of the
 *     Hessenberg least-squares problem; the modified Gram-Schmidt variant it names as
 *     the alternative to CGS, selected by or_gmres_args.ortho);
 *   - Section 3 ("CB-GMRES": basis stored in a compact format, all arithmetic FP64, the
 *     basis decompressed before each product with it in Fig. 1);
 *   - Section 4.2 (memory accessor; fixed-point formats with the per-vector scale
 *     sigma_j = (||v_j||_inf / ||v_j||_2) / max_intxx, applied as a post-multiplication
 *     by diag(Sigma) on every access);
 *   - Section 5.2 (explicit residual computed when the recurrence residual signals
 *     convergence; iteration continues with the updated residual otherwise).
 *
 * Readings taken where the paper is silent (each also listed in the design notes):
 *   R1  eta (re-orthogonalisation threshold) is not given: 1/sqrt(2) in conditional
 *       mode; the default mode re-orthogonalises always (one extra CGS pass).
 *   R2  the second clause of Fig. 1's breakdown test is read as a breakdown test
 *       !(h_{j+1,j} > eps_bd * omega); literal_fig1 = 1 restores the printed clause.
 *   R3  the division v := w / h_{j+1,j} (Fig. 1, first vector and basis extension) is a multiplication by the
 *       FP64 reciprocal 1/h, so that the stored codes are a fixed function of w.
 *   R4  "stored as v_j / sigma_j" (Section 4.2): q_i = clamp(rint(v_i / sigma_j)) with
 *       v = w / ||w||_2 normalised, sigma_j = max_i |v_i| / max_int (equal to the printed
 *       formula in exact arithmetic), 1/sigma_j applied as a multiplication, rint in
 *       round-to-nearest-even, clamp to [-max_int, max_int].
 *   R5  BF16 / FP8-e4m3 basis (not in the paper): per-vector power-of-two scale
 *       s = 2^e with e the smallest integer such that max|v| <= F_max * 2^e (F_max = 1
 *       for bf16, 448 for e4m3), code = RN_target(RN_fp32(v_i * 2^-e)); the FP32 step is
 *       part of the definition; e4m3 saturates to +-448.
 *   R6  f16 is a single round-to-nearest-even of the FP64 value (no scale), as a plain
 *       IEEE cast (Section 4.2 lists float16 without scaling).
 *   R7  iterations = Arnoldi steps (sparse products of Fig. 1's Arnoldi step); maxit caps them.
 *   R8  ||b|| = 0 returns x = 0 (exact solution) with zero iterations.
 *   R19 the order of the terms of an inner product is not given: index order within
 *       fixed blocks of OR_DOT_BLOCK terms, then the block sums in block order (the
 *       result does not depend on how many threads run the blocks).
 */
#ifndef CBG_ORACLE_H
#define CBG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage formats of the Krylov basis */
enum { OR_F64 = 0, OR_F32 = 1, OR_F16 = 2, OR_BF16 = 3, OR_E4M3 = 4, OR_I32 = 5, OR_I16 = 6 };
/* preconditioners (right preconditioning, Fig. 1) */
enum { OR_PC_NONE = 0, OR_PC_JACOBI = 1, OR_PC_SPAI = 2,
       OR_PC_BJ4 = 3 /* block-Jacobi, blocks of 4 consecutive rows (Section 5.5) */ };
/* re-orthogonalisation modes (Fig. 1) */
enum { OR_REORTH_ALWAYS = 0, OR_REORTH_CONDITIONAL = 1, OR_REORTH_NEVER = 2 };
/* orthogonalisation: classical Gram-Schmidt as Fig. 1 prints it, or the modified
 * Gram-Schmidt variant Section 2 mentions (each coefficient taken against w as already
 * reduced by the columns before it) */
enum { OR_ORTHO_CGS = 0, OR_ORTHO_MGS = 1 };
/* status codes */
enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_ERR_ARG = -1, OR_ERR_NONFINITE = -2 };

/* ---- scalar codec (exact definitions; no scale) ---------------------------------- */
uint16_t or_f64_to_f16(double x);   /* IEEE binary16, RNE, subnormals, overflow -> inf */
double   or_f16_to_f64(uint16_t h);
uint16_t or_f32_to_bf16(float x);   /* bfloat16, RNE, overflow -> inf                 */
double   or_bf16_to_f64(uint16_t b);
uint8_t  or_f32_to_e4m3(float x);   /* OCP FP8 E4M3 (no inf), RNE, saturate to 448    */
double   or_e4m3_to_f64(uint8_t c);
int      or_format_bytes(int fmt);
void or_vec_f64_to_f16(int64_t n, const double* x, uint16_t* out);
void or_vec_f16_to_f64(int64_t n, const uint16_t* c, double* out);
void or_vec_f32_to_bf16(int64_t n, const float* x, uint16_t* out);
void or_vec_bf16_to_f64(int64_t n, const uint16_t* c, double* out);
void or_vec_f32_to_e4m3(int64_t n, const float* x, uint8_t* out);
void or_vec_e4m3_to_f64(int64_t n, const uint8_t* c, double* out);

/* ---- vector codec (Section 4.2) ----------------------------------------------------
 * Encode a normalised vector v (FP64, length n) whose largest magnitude is vmax.
 * codes: n elements of or_format_bytes(fmt) bytes.  *scale receives the per-vector
 * factor (sigma for int formats, 2^e for bf16/e4m3, 1 otherwise).  Returns 0 or
 * OR_ERR_ARG. */
int or_encode(int fmt, int64_t n, const double* v, double vmax, void* codes, double* scale);
int or_decode(int fmt, int64_t n, const void* codes, double scale, double* out);

/* ---- threads ---------------------------------------------------------------------
 * Threads of the parallel loops (a build with OpenMP; 1 otherwise).  Results do not
 * depend on the count. */
void or_set_threads(int t);
int  or_get_threads(void);

/* ---- building blocks ------------------------------------------------------------- */
#define OR_DOT_BLOCK 4096
void   or_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
               const double* x, double* y);              /* y = A x, row sums in CSR order */
double or_dot(int64_t n, const double* a, const double* b); /* blocked sum (R19)        */
/* one Gram-Schmidt pass of w against the ncols columns of V (n x ncols, column-major):
 * coefficients c (ncols), w reduced in place; ortho = OR_ORTHO_CGS or OR_ORTHO_MGS */
void   or_gram_schmidt_pass(int64_t n, const double* V, int64_t ncols, int ortho, double* w,
                            double* c);

/* ---- GMRES(m) (Fig. 1 with Section 5.2's explicit-residual recheck) --------------- */
typedef struct {
    /* inputs */
    int32_t m;              /* restart length (basis dimension)                     */
    int32_t fmt;            /* OR_F64 ... OR_I16                                    */
    int32_t precond;        /* OR_PC_*                                              */
    int32_t reorth;         /* OR_REORTH_*                                          */
    int32_t literal_fig1;   /* 1: Fig. 1's breakdown clause literally (R2)       */
    int32_t adapt;          /* 1: adaptive basis format (reading R15)              */
    double  eta;            /* conditional re-orthogonalisation threshold          */
    double  eps_bd;         /* breakdown threshold on h_{j+1,j} / omega            */
    double  tol;            /* tau                                                  */
    int64_t maxit;          /* cap on Arnoldi steps                                 */
    const double* pvals;    /* SPAI values on A's pattern (precond == OR_PC_SPAI)  */
    /* optional outputs (NULL to skip) */
    double* H1;             /* (m+1) x m column-major raw Hessenberg, first cycle  */
    double* V1;             /* n x (m+1) column-major decoded basis, first cycle   */
    double* hist;           /* recurrence residual |g_{j+1}| / ||b|| per step      */
    int64_t hist_cap;
    double* tres;           /* true residual / ||b|| at the start of each cycle    */
    int64_t tres_cap;
    /* outputs */
    int64_t iters, cycles, reorths, k1, nhist, ntres;
    double  true_relres, est_relres;
    int32_t status, pad1;
    double  adapt_gap;      /* promotion threshold of adapt                         */
    int32_t fmt_final;      /* out: basis format of the last cycle                  */
    int32_t promotions;     /* out: format promotions                               */
    int32_t ortho;          /* OR_ORTHO_* (CGS by default)                          */
    int32_t pad2;
} or_gmres_args;

int or_gmres(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             const double* b, double* x /* in: x0, out: x */, or_gmres_args* a);

/* ---- learned SPAI preconditioner: per-row MLP (7 -> 64 -> 64 -> 7), FP64 ---------- */
int or_mlp_forward(int64_t rows, const double* feat /* rows x 7 */,
                   const double* W1, const double* b1, const double* W2, const double* b2,
                   const double* W3, const double* b3, double* out /* rows x 7 */,
                   double* act1 /* rows x 64 or NULL */, double* act2 /* rows x 64 or NULL */);
int or_mlp_backward(int64_t rows, const double* feat, const double* W1, const double* b1,
                    const double* W2, const double* b2, const double* W3, const double* b3,
                    const double* gout /* rows x 7: dL/dout */,
                    double* gW1, double* gb1, double* gW2, double* gb2, double* gW3, double* gb3);

/* ---- learned SPAI: statistics of (r, e) pairs and the loss (no counterpart in the paper:
 * parity unpinned by the paper; pinned to finite differences and direct evaluation) ----
 * slot[p] in 0..6 is the stencil position of nonzero p (-z,-y,-x,centre,+x,+y,+z for a
 * 3D 7-point pattern with line stride sx and plane stride sxy).  For one pair with
 * weight wgt = 1/||e||^2:  G_i[k][l] += wgt r_{nb(i,k)} r_{nb(i,l)},  c_i[k] += wgt e_i
 * r_{nb(i,k)},  d_i += wgt e_i^2  (G: rows x 49, c: rows x 7, d: rows). */
int or_spai_slots(int64_t n, const int32_t* rowptr, const int32_t* col, int64_t sx, int64_t sxy,
                  int8_t* slot);
int or_spai_accumulate(int64_t n, const int32_t* rowptr, const int32_t* col, const int8_t* slot,
                       const double* r, const double* e, double wgt, double* G, double* c, double* d);
/* loss = (1/npairs) sum_i [p_i^T G_i p_i - 2 p_i^T c_i + d_i] with p_i[k] = out[i][k] / diag_i
 * for existing slots; gout[i][k] = dloss/dout[i][k]. */
double or_spai_loss(int64_t n, const int32_t* rowptr, const int8_t* slot, const double* out,
                    const double* diag, const double* G, const double* c, const double* d,
                    double npairs, double* gout);

#ifdef __cplusplus
}
#endif
#endif
