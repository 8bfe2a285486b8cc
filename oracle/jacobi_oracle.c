/*
 * Jacobi3D oracle: a plain, slow, obviously correct CPU implementation of
 * the iteration the GPU library computes.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load this library. It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes (paper: Section II-A, Fig. 1 and Fig. 3 -- every iteration
 * the halos of the previous iteration are exchanged, then the whole block is
 * updated; Section III-C -- two separate copies of the grid, one read and one
 * written per iteration). The paper does not print the update formula; the
 * readings taken here are:
 *   - 7-point averaging: new value = (c + xm + xp + ym + yp + zm + zp) / 7,
 *     c the cell, xm/xp its -x/+x neighbours and so on;
 *   - the grid is NOT decomposed here: decomposition into blocks, halo pack,
 *     exchange and unpack are implementation details that do not change the
 *     result, so the oracle iterates one (nx+2)(ny+2)(nz+2) array whose
 *     one-cell ghost frame holds fixed Dirichlet values bc[0..5] for the
 *     planes outside the -x, +x, -y, +y, -z, +z faces;
 *   - x is the contiguous axis; interior arrays are x fastest:
 *     cell (i, j, k) is element i + nx*(j + ny*k).
 *
 * Three ways to round the average are provided:
 *   ORC_RULE_SEQ   : binary64, sum taken left to right in the order
 *                    c, xm, xp, ym, yp, zm, zp, each addition rounded to
 *                    nearest even, then one correctly rounded division by 7.
 *   ORC_RULE_EXACT : binary64, the exact sum of the seven values divided by 7
 *                    and rounded once to nearest even (the correctly rounded
 *                    mean). Computed with an exact fixed-point accumulator.
 *   orc_jacobi_f32 : binary32 storage and arithmetic, same order as SEQ.
 *
 * The residual is rho(u) = sqrt( sum over interior cells of L^2 ), with
 * L = xm + xp + ym + yp + zm + zp - 6c evaluated exactly and rounded once to
 * binary64, squared in binary64 and summed with Neumaier's compensated sum.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -fno-fast-math [-fopenmp].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

#define ORC_RULE_SEQ 0
#define ORC_RULE_EXACT 1

/* Planted mistakes for the pin tests' mutation check (tests/test_oracle_mutants.py).
 * The oracle is always built with ORC_MUTANT == 0; a test builds a copy with a
 * nonzero value into a temporary directory and checks that some pin fails. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

/* ------------------------------------------------------------------ */
/* Ghosted global grid                                                 */
/* ------------------------------------------------------------------ */

static size_t gi(int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny)
{
    return (size_t)(i + 1) + (size_t)(nx + 2) * ((size_t)(j + 1) + (size_t)(ny + 2) * (size_t)(k + 1));
}

static size_t ghosted_cells(int64_t nx, int64_t ny, int64_t nz)
{
    return (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
}

/* Fill the six ghost planes with the Dirichlet values (edges and corners of
 * the ghost frame are never read by a 7-point stencil and stay 0). */
static void set_ghosts_f64(double *g, int64_t nx, int64_t ny, int64_t nz, const double bc[6])
{
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j) {
            g[gi(-1, j, k, nx, ny)] = bc[ORC_MUTANT == 2 ? 1 : 0];
            g[gi(nx, j, k, nx, ny)] = bc[ORC_MUTANT == 2 ? 0 : 1];
        }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < nx; ++i) {
            g[gi(i, -1, k, nx, ny)] = bc[2];
            g[gi(i, ny, k, nx, ny)] = bc[3];
        }
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            g[gi(i, j, -1, nx, ny)] = bc[4];
            g[gi(i, j, nz, nx, ny)] = bc[5];
        }
}

static void set_ghosts_f32(float *g, int64_t nx, int64_t ny, int64_t nz, const double bc[6])
{
    float b[6];
    for (int f = 0; f < 6; ++f) b[f] = (float)bc[f];
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j) {
            g[gi(-1, j, k, nx, ny)] = b[0];
            g[gi(nx, j, k, nx, ny)] = b[1];
        }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < nx; ++i) {
            g[gi(i, -1, k, nx, ny)] = b[2];
            g[gi(i, ny, k, nx, ny)] = b[3];
        }
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            g[gi(i, j, -1, nx, ny)] = b[4];
            g[gi(i, j, nz, nx, ny)] = b[5];
        }
}

/* ------------------------------------------------------------------ */
/* Exact accumulator for sums of binary64 values with small integer    */
/* weights. Bit p of the accumulator has weight 2^(p - 1074), so every  */
/* finite double is an integer multiple of bit 0.                      */
/* ------------------------------------------------------------------ */

#define XWORDS 72 /* 72 x 32 = 2304 bits, enough for 2^1024 * 7 * 7 */

typedef struct {
    uint32_t w[XWORDS];
} xacc;

/* add m * 2^pos (m < 2^60) to a magnitude accumulator */
static void xacc_add(xacc *a, uint64_t m, int pos)
{
    int q = pos >> 5;
    int sh = pos & 31;
    /* m << sh spans at most 92 bits: three 32-bit words */
    uint64_t lo = m << sh;                          /* bits 0..63 of the shifted value */
    uint64_t hi = sh ? (m >> (64 - sh)) : 0;        /* bits 64..91 */
    uint32_t part[3] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi};
    uint64_t carry = 0;
    for (int t = 0; t < 3; ++t) {
        uint64_t s = (uint64_t)a->w[q + t] + part[t] + carry;
        a->w[q + t] = (uint32_t)s;
        carry = s >> 32;
    }
    for (int t = q + 3; carry && t < XWORDS; ++t) {
        uint64_t s = (uint64_t)a->w[t] + carry;
        a->w[t] = (uint32_t)s;
        carry = s >> 32;
    }
}

/* add w * v (w a small integer, |w| <= 7) to the positive or negative part */
static void xacc_add_double(xacc *pos_part, xacc *neg_part, double v, int w)
{
    uint64_t bits;
    memcpy(&bits, &v, 8);
    int neg = (int)(bits >> 63);
    int e = (int)((bits >> 52) & 0x7FF);
    uint64_t frac = bits & ((1ULL << 52) - 1);
    uint64_t m;
    int p;
    if (e == 0) {           /* zero or subnormal: frac * 2^-1074 */
        m = frac;
        p = 0;
    } else {                /* normal: (2^52 + frac) * 2^(e - 1075) */
        m = frac | (1ULL << 52);
        p = e - 1;
    }
    if (m == 0) return;
    if (w < 0) {
        neg = !neg;
        w = -w;
    }
    m *= (uint64_t)w;
    xacc_add(neg ? neg_part : pos_part, m, p);
}

/* |P - N| into out, returns the sign (1 if negative) */
static int xacc_diff(const xacc *P, const xacc *N, xacc *out)
{
    int cmp = 0;
    for (int t = XWORDS - 1; t >= 0 && cmp == 0; --t) {
        if (P->w[t] > N->w[t]) cmp = 1;
        else if (P->w[t] < N->w[t]) cmp = -1;
    }
    const xacc *big = (cmp >= 0) ? P : N;
    const xacc *small = (cmp >= 0) ? N : P;
    int64_t borrow = 0;
    for (int t = 0; t < XWORDS; ++t) {
        int64_t d = (int64_t)big->w[t] - (int64_t)small->w[t] - borrow;
        borrow = d < 0;
        out->w[t] = (uint32_t)(d + (borrow ? (1LL << 32) : 0));
    }
    return cmp < 0;
}

static int xacc_bit(const xacc *a, int p)
{
    return (int)((a->w[p >> 5] >> (p & 31)) & 1u);
}

/* Round (S / d) * 2^-1074 to the nearest binary64, ties to even, where S is
 * the magnitude in `a` and d is 1 or 7. The division is ordinary long
 * division over the 32-bit words; r is the final remainder. */
static double xacc_round_div(xacc *a, uint32_t d, int negative)
{
    xacc q;
    uint64_t r = 0;
    for (int t = XWORDS - 1; t >= 0; --t) {
        uint64_t cur = (r << 32) | a->w[t];
        uint64_t qt = (d == 7) ? cur / 7u : cur;
        q.w[t] = (uint32_t)qt;
        r = cur - qt * d;
    }
    int top = -1;
    for (int t = XWORDS - 1; t >= 0 && top < 0; --t)
        if (q.w[t]) top = t * 32 + 31 - __builtin_clz(q.w[t]);
    uint64_t mant;
    int shift;
    int up;
    if (top < 0) {
        /* quotient below 2^-1074: only the fraction r/d remains */
        mant = 0;
        shift = 0;
        up = (2 * r > d);
    } else {
        shift = top > 52 ? top - 52 : 0;
        mant = 0;
        for (int p = top; p >= shift; --p) mant = (mant << 1) | (uint64_t)xacc_bit(&q, p);
        if (shift > 0) {
            int rbit = xacc_bit(&q, shift - 1);
            /* sticky: any quotient bit below shift-1, or a nonzero remainder */
            int sticky = (r != 0);
            int below = shift - 1; /* bits 0 .. below-1 */
            int wfull = below >> 5;
            for (int t = 0; t < wfull && !sticky; ++t) sticky = (q.w[t] != 0);
            if (!sticky && (below & 31)) sticky = (q.w[wfull] & ((1u << (below & 31)) - 1u)) != 0;
            up = rbit && (sticky || (mant & 1));
        } else {
            /* the tail is r/d of one unit of 2^-1074 */
            up = (2 * r > d) || (2 * r == d && (mant & 1));
        }
    }
    if (ORC_MUTANT == 4) up = 0;
    mant += (uint64_t)up;
    double v = ldexp((double)mant, shift - 1074);
    return negative ? -v : v;
}

/* The correctly rounded mean of seven doubles. An exact zero gives +0.0. */
static double exact_mean7(const double v[7])
{
    xacc P, N, S;
    memset(&P, 0, sizeof P);
    memset(&N, 0, sizeof N);
    for (int t = 0; t < 7; ++t) xacc_add_double(&P, &N, v[t], 1);
    int neg = xacc_diff(&P, &N, &S);
    double r = xacc_round_div(&S, 7, neg);
    return r == 0.0 ? 0.0 : r;
}

/* xm + xp + ym + yp + zm + zp - 6c, exact, rounded once to binary64. */
static double exact_laplacian(double c, const double nb[6])
{
    xacc P, N, S;
    memset(&P, 0, sizeof P);
    memset(&N, 0, sizeof N);
    for (int t = 0; t < 6; ++t) xacc_add_double(&P, &N, nb[t], 1);
    xacc_add_double(&P, &N, c, ORC_MUTANT == 5 ? 6 : -6);
    int neg = xacc_diff(&P, &N, &S);
    double r = xacc_round_div(&S, 1, neg);
    return r == 0.0 ? 0.0 : r;
}

/* exposed for the exactness tests */
double orc_exact_mean7(const double *v) { return exact_mean7(v); }
double orc_exact_laplacian(double c, const double *nb) { return exact_laplacian(c, nb); }

/* ------------------------------------------------------------------ */
/* Iteration                                                           */
/* ------------------------------------------------------------------ */

static void sweep_f64(const double *src, double *dst, int64_t nx, int64_t ny, int64_t nz, int rule)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double c = src[gi(i, j, k, nx, ny)];
                double xm = src[gi(i - 1, j, k, nx, ny)];
                double xp = src[gi(i + 1, j, k, nx, ny)];
                double ym = (ORC_MUTANT == 3) ? src[gi(i - 1, j, k, nx, ny)] : src[gi(i, j - 1, k, nx, ny)];
                double yp = src[gi(i, j + 1, k, nx, ny)];
                double zm = src[gi(i, j, k - 1, nx, ny)];
                double zp = src[gi(i, j, k + 1, nx, ny)];
                double out;
                if (rule == ORC_RULE_SEQ) {
                    double s = c;
                    if (ORC_MUTANT == 7) {
                        s = s + (xm + xp);
                    } else {
                        s = s + xm;
                        s = s + xp;
                    }
                    s = s + ym;
                    s = s + yp;
                    s = s + zm;
                    if (ORC_MUTANT != 1) s = s + zp;
                    if (ORC_MUTANT == 8) out = s * (1.0 / 7.0);
                    else out = s / (ORC_MUTANT == 6 ? 6.0 : 7.0);
                } else {
                    double v[7] = {c, xm, xp, ym, yp, zm, zp};
                    out = exact_mean7(v);
                }
                dst[gi(i, j, k, nx, ny)] = out;
            }
}

/* Run n_iters Jacobi iterations from the interior u0 (x fastest) with the
 * Dirichlet ghost values bc[6]; write the final interior to out. */
int orc_jacobi_f64(int64_t nx, int64_t ny, int64_t nz, const double *bc, const double *u0,
                   int64_t n_iters, double *out, int rule)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_iters < 0 || !bc || !u0 || !out) return ORC_EINVAL;
    if (rule != ORC_RULE_SEQ && rule != ORC_RULE_EXACT) return ORC_EINVAL;
    size_t n = ghosted_cells(nx, ny, nz);
    double *a = (double *)calloc(n, sizeof(double));
    double *b = (double *)calloc(n, sizeof(double));
    if (!a || !b) {
        free(a);
        free(b);
        return ORC_ENOMEM;
    }
    set_ghosts_f64(a, nx, ny, nz, bc);
    set_ghosts_f64(b, nx, ny, nz, bc);
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) a[gi(i, j, k, nx, ny)] = u0[i + nx * (j + ny * k)];
    for (int64_t it = 0; it < n_iters; ++it) {
        sweep_f64(a, b, nx, ny, nz, rule);
        double *t = a;
        a = b;
        b = t;
    }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) out[i + nx * (j + ny * k)] = a[gi(i, j, k, nx, ny)];
    free(a);
    free(b);
    return ORC_OK;
}

/* binary32 storage and arithmetic; bc are rounded to binary32 first. */
int orc_jacobi_f32(int64_t nx, int64_t ny, int64_t nz, const double *bc, const float *u0,
                   int64_t n_iters, float *out)
{
    if (nx < 1 || ny < 1 || nz < 1 || n_iters < 0 || !bc || !u0 || !out) return ORC_EINVAL;
    size_t n = ghosted_cells(nx, ny, nz);
    float *a = (float *)calloc(n, sizeof(float));
    float *b = (float *)calloc(n, sizeof(float));
    if (!a || !b) {
        free(a);
        free(b);
        return ORC_ENOMEM;
    }
    set_ghosts_f32(a, nx, ny, nz, bc);
    set_ghosts_f32(b, nx, ny, nz, bc);
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) a[gi(i, j, k, nx, ny)] = u0[i + nx * (j + ny * k)];
    for (int64_t it = 0; it < n_iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    float s = a[gi(i, j, k, nx, ny)];
                    s = s + a[gi(i - 1, j, k, nx, ny)];
                    s = s + a[gi(i + 1, j, k, nx, ny)];
                    s = s + a[gi(i, j - 1, k, nx, ny)];
                    s = s + a[gi(i, j + 1, k, nx, ny)];
                    s = s + a[gi(i, j, k - 1, nx, ny)];
                    s = s + a[gi(i, j, k + 1, nx, ny)];
                    b[gi(i, j, k, nx, ny)] = (ORC_MUTANT == 9) ? s * (1.0f / 7.0f) : s / 7.0f;
                }
        float *t = a;
        a = b;
        b = t;
    }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) out[i + nx * (j + ny * k)] = a[gi(i, j, k, nx, ny)];
    free(a);
    free(b);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Residual                                                            */
/* ------------------------------------------------------------------ */

/* Neumaier's compensated summation of one term into (s, c) */
static void neumaier(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

static int residual_ghosted(const double *g, int64_t nx, int64_t ny, int64_t nz, double *rho)
{
    /* one compensated partial sum per z-plane, combined in plane order, so the
     * result does not depend on the number of threads */
    double *ps = (double *)calloc((size_t)nz, sizeof(double));
    double *pc = (double *)calloc((size_t)nz, sizeof(double));
    if (!ps || !pc) {
        free(ps);
        free(pc);
        return ORC_ENOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k) {
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                double nb[6] = {g[gi(i - 1, j, k, nx, ny)], g[gi(i + 1, j, k, nx, ny)],
                                g[gi(i, j - 1, k, nx, ny)], g[gi(i, j + 1, k, nx, ny)],
                                g[gi(i, j, k - 1, nx, ny)], g[gi(i, j, k + 1, nx, ny)]};
                double L = exact_laplacian(g[gi(i, j, k, nx, ny)], nb);
                neumaier(&s, &c, L * L);
            }
        ps[k] = s;
        pc[k] = c;
    }
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < nz; ++k) {
        neumaier(&s, &c, ps[k]);
        neumaier(&s, &c, pc[k]);
    }
    *rho = sqrt(s + c);
    free(ps);
    free(pc);
    return ORC_OK;
}

int orc_residual_f64(int64_t nx, int64_t ny, int64_t nz, const double *bc, const double *u, double *rho)
{
    if (nx < 1 || ny < 1 || nz < 1 || !bc || !u || !rho) return ORC_EINVAL;
    double *g = (double *)calloc(ghosted_cells(nx, ny, nz), sizeof(double));
    if (!g) return ORC_ENOMEM;
    set_ghosts_f64(g, nx, ny, nz, bc);
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) g[gi(i, j, k, nx, ny)] = u[i + nx * (j + ny * k)];
    int rc = residual_ghosted(g, nx, ny, nz, rho);
    free(g);
    return rc;
}

/* residual of a binary32 grid: values (and bc rounded to binary32) are
 * widened exactly to binary64 and the same definition is applied */
int orc_residual_f32(int64_t nx, int64_t ny, int64_t nz, const double *bc, const float *u, double *rho)
{
    if (nx < 1 || ny < 1 || nz < 1 || !bc || !u || !rho) return ORC_EINVAL;
    double b[6];
    for (int f = 0; f < 6; ++f) b[f] = (double)(float)bc[f];
    double *g = (double *)calloc(ghosted_cells(nx, ny, nz), sizeof(double));
    if (!g) return ORC_ENOMEM;
    set_ghosts_f64(g, nx, ny, nz, b);
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) g[gi(i, j, k, nx, ny)] = (double)u[i + nx * (j + ny * k)];
    int rc = residual_ghosted(g, nx, ny, nz, rho);
    free(g);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
