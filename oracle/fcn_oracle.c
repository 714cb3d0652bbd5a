/*
 * fcn_oracle.c -- plain FP64 CPU oracle of the FCN z-step (Ma & Lin,
 * arXiv:1507.05988, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code; the CUDA library never does.  It is
 * written to be read against the paper: every loop follows the order in which
 * Sec. 3 states the method, with no blocking, fusion or reordering.
 *
 * Readings of the paper taken here (the paper is ambiguous or garbled at
 * these places):
 *   R1  c_j and f_j (Sec. 3, coefficients of Eq. (matrix1)) carry the factor
 *       (1 + 1/(2j)), which is what Eqs. (diff2)-(diff3) give for the
 *       A_{j+1} entries; the printed (1 - 1/(2j)) is kept behind
 *       ORC_PRINTED_CJ only so the tests can show that it is rejected.
 *   R2  The plasma term of Eq. (nonlinearpart) uses omega_pe^2/omega0^2
 *       = rho/rho_c (the printed omega_pe^2/omega0 is not dimensionless):
 *       N_plasma = -i k0/(2 n0^2) rho/rho_c.
 *   R3  rho follows Eq. (ionization) with beta_K/(K hbar omega0) written as
 *       sigma_K rho_nt and rho_at := rho_nt, i.e.
 *       d rho/d tau = sigma_K I^K (rho_nt - rho).
 *   R4  Within one nonlinear half step (Eq. (Anhalf)) N is frozen at the
 *       field entering that half step; rho is integrated by RK4 (Sec. 3.2)
 *       from rho(tau_min) = 0 using the intensity of the pre-update row, with
 *       the RK4 midpoint intensity taken as the mean of the two neighbours.
 *   R5  Grid: dr = R/(Nr-1) with the Dirichlet node at m = Nr-1 (Eq. (bound));
 *       dtau = T/Nt, tau_p = -T/2 + p dtau, periodic in tau; omega_q = 2 pi q
 *       /(Nt dtau) for q < Nt/2 and 2 pi (q - Nt)/(Nt dtau) otherwise.
 *   R6  The forward transform is exp(-2 pi i p q / Nt), unnormalised; the
 *       inverse carries 1/Nt (Eq. (antifourier)).
 *   R9  Cartesian transverse grid (Sec. 2 names Delta_perp = d^2/dx^2 +
 *       d^2/dy^2 but Sec. 3 discretises only the radial operator): each axis
 *       takes the second difference of Eq. (diff2) with the Crank-Nicolson
 *       average of Eq. (diff1); the walls carry A = 0 (Eq. (bound) at
 *       r = max, on all four sides).  The two-dimensional system is not
 *       tridiagonal, so the linear step is the product of the two 1-D
 *       Cayley factors, x first, then y (the Peaceman-Rachford alternating
 *       direction form); the factors commute, and the product differs from
 *       the unsplit 2-D Crank-Nicolson step by O(dz^3) per step, the order
 *       of the Strang split itself.  The dispersion term goes into the y
 *       factor whole, so a transversely uniform field sees exactly the
 *       radial scheme's factor (1 + i delta_q)/(1 - i delta_q).
 */
#include "fcn_oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 values (SI). */
#define ORC_C_LIGHT 299792458.0
#define ORC_HBAR    1.054571817e-34
#define ORC_EPS0    8.8541878128e-12
#define ORC_M_E     9.1093837015e-31
#define ORC_Q_E     1.602176634e-19
#define ORC_PI      3.14159265358979323846

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Derived constants                                                   */
/* ------------------------------------------------------------------ */

/* Carrier wave number k0 = 2 pi n0 / lambda0 (Sec. 2). */
double orc_k0(const orc_problem *pb) { return 2.0 * ORC_PI * pb->n0 / pb->lambda0; }

/* Carrier angular frequency omega0 = 2 pi c / lambda0 (Sec. 2). */
double orc_omega0(const orc_problem *pb) { return 2.0 * ORC_PI * ORC_C_LIGHT / pb->lambda0; }

/* Critical plasma density rho_c = eps0 m_e omega0^2 / q_e^2, the density at
 * which omega_pe (Sec. 2, below Eq. (plasmasource)) equals omega0 (reading R2). */
double orc_rho_c(const orc_problem *pb)
{
    double w0 = orc_omega0(pb);
    return ORC_EPS0 * ORC_M_E * w0 * w0 / (ORC_Q_E * ORC_Q_E);
}

/* MPI loss coefficient beta_K = K hbar omega0 sigma_K rho_nt, so that the
 * rate of Eq. (ionization) is sigma_K I^K (rho_nt - rho) (reading R3). */
double orc_beta_k(const orc_problem *pb)
{
    return (double)pb->K * ORC_HBAR * orc_omega0(pb) * pb->sigma_k * pb->rho_nt;
}

/* Angular frequency of FFT bin q (reading R5). */
double orc_omega(const orc_problem *pb, int q)
{
    double dtau = pb->t_window / pb->nt;
    int qq = (q < pb->nt / 2) ? q : q - pb->nt;
    return 2.0 * ORC_PI * (double)qq / (pb->nt * dtau);
}

static double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

/* ------------------------------------------------------------------ */
/* FFT along tau (Sec. 3.1, first and third loop)                     */
/* ------------------------------------------------------------------ */

/* In-place iterative radix-2 Cooley-Tukey transform of n interleaved complex
 * values.  inverse = 0: X_q = sum_p x_p exp(-2 pi i p q / n).
 * inverse = 1: x_p = (1/n) sum_q X_q exp(+2 pi i p q / n).
 * Returns -1 if n is not a power of two. */
int orc_fft(double *xd, int n, int inverse)
{
    if (n < 1 || (n & (n - 1)) != 0) return -1;
    cplx *x = (cplx *)xd;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    double sgn = inverse ? 1.0 : -1.0;
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double ang = sgn * 2.0 * ORC_PI * (double)k / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (int s = 0; s < n; s += len) {
                cplx u = x[s + k];
                cplx v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
    if (inverse) {
        double inv = 1.0 / (double)n;
        for (int i = 0; i < n; ++i) x[i] *= inv;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Tridiagonal "chasing" solve (Sec. 3.1, remark after the loops)     */
/* ------------------------------------------------------------------ */

/* Thomas algorithm without pivoting for
 *   a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j,  j = 0..n-1
 * (a_0 and c_{n-1} are ignored).  All arrays interleaved complex.
 * Returns -1 on a zero pivot. */
int orc_thomas(int n, const double *ad, const double *bd, const double *cd,
               const double *dd, double *xd)
{
    const cplx *a = (const cplx *)ad, *b = (const cplx *)bd, *c = (const cplx *)cd;
    const cplx *d = (const cplx *)dd;
    cplx *x = (cplx *)xd;
    cplx *cp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    cplx *dp = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!cp || !dp) { free(cp); free(dp); return -2; }
    cplx piv = b[0];
    if (piv == 0) { free(cp); free(dp); return -1; }
    cp[0] = c[0] / piv;
    dp[0] = d[0] / piv;
    for (int j = 1; j < n; ++j) {
        piv = b[j] - a[j] * cp[j - 1];
        if (piv == 0) { free(cp); free(dp); return -1; }
        cp[j] = (j < n - 1) ? c[j] / piv : 0;
        dp[j] = (d[j] - a[j] * dp[j - 1]) / piv;
    }
    x[n - 1] = dp[n - 1];
    for (int j = n - 2; j >= 0; --j) x[j] = dp[j] - cp[j] * x[j + 1];
    free(cp);
    free(dp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Crank-Nicolson matrices (Eqs. (diff1)-(diff3), (bound), (matrix))  */
/* ------------------------------------------------------------------ */

/* Fills the six diagonals of M_abc^q (a, b, c) and M_def^q (d, e, f) for
 * frequency bin q, each nr interleaved complex values.
 * With s = dz/(4 k0 dr^2) and delta_q = k'' omega_q^2 dz / 4:
 *   row 0      : b = 1 + 4is - i delta, c = -4is, e = 1 - 4is + i delta, f = 4is
 *   1<=j<=nr-2 : a = -is(1 - 1/2j), b = 1 + 2is - i delta, c = -is(1 + 1/2j)
 *                d =  is(1 - 1/2j), e = 1 - 2is + i delta, f =  is(1 + 1/2j)
 *   row nr-1   : b = 1, a = c = d = e = f = 0       (A = 0 at r = R)
 * (delta_q = 0 under ORC_EXACT_DISPERSION, whose exact factor cn_column
 * applies after the solve.)
 * The row-0 entries come from the r -> 0 limit Delta_perp -> 2 d^2/dr^2 with
 * the mirror point A_{-1} = A_1 (dA/dr = 0 at r = 0, Eq. (bound)). */
void orc_cn_coeffs(const orc_problem *pb, double dz, int q,
                   double *ad, double *bd, double *cd,
                   double *dd, double *ed, double *fd)
{
    int nr = pb->nr;
    cplx *a = (cplx *)ad, *b = (cplx *)bd, *c = (cplx *)cd;
    cplx *d = (cplx *)dd, *e = (cplx *)ed, *f = (cplx *)fd;
    double dr = pb->r_max / (double)(nr - 1);
    double k0 = orc_k0(pb);
    double s = (pb->flags & ORC_DIFFRACTION) ? dz / (4.0 * k0 * dr * dr) : 0.0;
    double w = orc_omega(pb, q);
    /* with ORC_EXACT_DISPERSION the CN system carries diffraction alone */
    double delta = ((pb->flags & ORC_DISPERSION) && !(pb->flags & ORC_EXACT_DISPERSION))
                       ? pb->k2 * w * w * dz / 4.0 : 0.0;

    a[0] = 0;
    b[0] = 1.0 + I * (4.0 * s) - I * delta;
    c[0] = -I * (4.0 * s);
    d[0] = 0;
    e[0] = 1.0 - I * (4.0 * s) + I * delta;
    f[0] = I * (4.0 * s);
    for (int j = 1; j <= nr - 2; ++j) {
        double lo = 1.0 - 1.0 / (2.0 * j);
        double hi = (pb->flags & ORC_PRINTED_CJ) ? lo : 1.0 + 1.0 / (2.0 * j);
        a[j] = -I * s * lo;
        b[j] = 1.0 + I * (2.0 * s) - I * delta;
        c[j] = -I * s * hi;
        d[j] = I * s * lo;
        e[j] = 1.0 - I * (2.0 * s) + I * delta;
        f[j] = I * s * hi;
    }
    a[nr - 1] = 0;
    b[nr - 1] = 1.0;
    c[nr - 1] = 0;
    d[nr - 1] = 0;
    e[nr - 1] = 0;
    f[nr - 1] = 0;
}

/* ------------------------------------------------------------------ */
/* Plasma density along tau (Eq. (ionization), RK4 of Sec. 3.2)       */
/* ------------------------------------------------------------------ */

/* d rho / d tau = sigma_K I^K (rho_nt - rho)   (reading R3) */
static double rho_rate(const orc_problem *pb, double intensity, double rho)
{
    return pb->sigma_k * ipow(intensity, pb->K) * (pb->rho_nt - rho);
}

/* Integrates rho along one row with classic RK4, step dtau, from
 * rho(tau_min) = 0.  intensity[p] = |A_{m,p}|^2 of the row entering the half
 * step; the midpoint intensity is the mean of its neighbours (reading R4). */
void orc_rho_row(const orc_problem *pb, const double *intensity, double *rho)
{
    double h = pb->t_window / pb->nt;
    rho[0] = 0.0;
    for (int p = 0; p + 1 < pb->nt; ++p) {
        double ia = intensity[p];
        double ib = intensity[p + 1];
        double im = 0.5 * (ia + ib);
        double r = rho[p];
        double k1 = rho_rate(pb, ia, r);
        double k2 = rho_rate(pb, im, r + 0.5 * h * k1);
        double k3 = rho_rate(pb, im, r + 0.5 * h * k2);
        double k4 = rho_rate(pb, ib, r + h * k3);
        rho[p + 1] = r + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }
}

/* ------------------------------------------------------------------ */
/* Nonlinear half step (Eqs. (nonlinearpart), (Anhalf), (Anhalf1))     */
/* ------------------------------------------------------------------ */

/* The operator N of Eq. (nonlinearpart) at intensity I and density rho:
 *   N = i (k0/n0) sum_j n_2j I^j - i k0/(2 n0^2) rho/rho_c - (beta_K/2) I^(K-1)
 * (readings R2, R3; the optional ORC_MPI_SAT factor multiplies the loss by
 * (1 - rho/rho_nt)). */
static cplx nl_operator(const orc_problem *pb, double intensity, double rho)
{
    double k0 = orc_k0(pb);
    double phase = 0.0, loss = 0.0;
    if (pb->flags & ORC_KERR) {
        double ij = 1.0;
        for (int j = 0; j < 4; ++j) {
            ij *= intensity;
            phase += (k0 / pb->n0) * pb->n2j[j] * ij;
        }
    }
    if (pb->flags & ORC_PLASMA)
        phase -= k0 / (2.0 * pb->n0 * pb->n0) * rho / orc_rho_c(pb);
    if (pb->flags & ORC_MPI) {
        loss = 0.5 * orc_beta_k(pb) * ipow(intensity, pb->K - 1);
        if (pb->flags & ORC_MPI_SAT) loss *= (1.0 - rho / pb->rho_nt);
    }
    return -loss + I * phase;
}

/* One nonlinear half step on one row: rho from the row as it enters
 * (orc_rho_row), then A_p <- A_p exp(h N(I_p, rho_p)) for p = 0..nt-1, with
 * h = dz/2.  rho (nt values) receives the density used. */
void orc_nl_half(const orc_problem *pb, double h, double *rowd, double *rho)
{
    int nt = pb->nt;
    cplx *row = (cplx *)rowd;
    double *inten = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!inten) {                    /* no memory: mark the row as failed */
        for (int p = 0; p < nt; ++p) {
            row[p] = NAN;
            rho[p] = NAN;
        }
        return;
    }
    for (int p = 0; p < nt; ++p) {
        double re = creal(row[p]), im = cimag(row[p]);
        inten[p] = re * re + im * im;
    }
    orc_rho_row(pb, inten, rho);
    for (int p = 0; p < nt; ++p) row[p] *= cexp(h * nl_operator(pb, inten[p], rho[p]));
    free(inten);
}

/* ------------------------------------------------------------------ */
/* Linear step (Sec. 3.1: three loops)                                 */
/* ------------------------------------------------------------------ */

/* Column q of the second loop: A~_{.,q} <- (M_abc^q)^{-1} M_def^q A~_{.,q}.
 * co: scratch of 8 nr complex values. */
static int cn_column(const orc_problem *pb, double dz, cplx *A, int q, cplx *co)
{
    int nr = pb->nr, nt = pb->nt;
    cplx *a = co, *b = co + nr, *c = co + 2 * nr, *d = co + 3 * nr;
    cplx *e = co + 4 * nr, *f = co + 5 * nr, *col = co + 6 * nr, *rhs = co + 7 * nr;
    orc_cn_coeffs(pb, dz, q, (double *)a, (double *)b, (double *)c,
                  (double *)d, (double *)e, (double *)f);
    for (int j = 0; j < nr; ++j) col[j] = A[(size_t)j * nt + q];
    /* rhs = M_def^q * A~_{.,q} */
    for (int j = 0; j < nr; ++j) {
        cplx v = e[j] * col[j];
        if (j > 0) v += d[j] * col[j - 1];
        if (j < nr - 1) v += f[j] * col[j + 1];
        rhs[j] = v;
    }
    int rc = orc_thomas(nr, (double *)a, (double *)b, (double *)c,
                        (double *)rhs, (double *)col);
    cplx ph = 1.0;
    if ((pb->flags & ORC_DISPERSION) && (pb->flags & ORC_EXACT_DISPERSION)) {
        /* exact dispersion over dz: dA~/dz = (i k''/2) omega^2 A~ from the
           -(i k''/2) d^2/dtau^2 term of Eq. (linearpart) */
        double w = orc_omega(pb, q);
        ph = cexp(I * (pb->k2 * w * w * dz / 2.0));
    }
    for (int j = 0; j < nr; ++j) A[(size_t)j * nt + q] = ph * col[j];
    return rc;
}

/* A <- F^{-1}( (M_abc^q)^{-1} M_def^q F(A) ) for the whole nr x nt field. */
int orc_linear_step(const orc_problem *pb, double dz, double *Ad)
{
    int nr = pb->nr, nt = pb->nt;
    cplx *A = (cplx *)Ad;
    /* first loop: forward transform of every row */
    for (int m = 0; m < nr; ++m)
        if (orc_fft((double *)(A + (size_t)m * nt), nt, 0)) return -1;
    /* second loop: one tridiagonal system per frequency */
    cplx *co = (cplx *)malloc(sizeof(cplx) * (size_t)nr * 8);
    if (!co) return -3;
    int rc = 0;
    for (int q = 0; q < nt && rc == 0; ++q) rc = cn_column(pb, dz, A, q, co);
    free(co);
    if (rc) return -2;
    /* third loop: inverse transform of every row */
    for (int m = 0; m < nr; ++m)
        if (orc_fft((double *)(A + (size_t)m * nt), nt, 1)) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* One Strang step (Eq. (nlseq)) and the serial driver (Sec. 3 end)    */
/* ------------------------------------------------------------------ */

/* A^{n+1} = exp(N dz/2) exp(D dz) exp(N dz/2) A^n.  rho (nr*nt, nullable)
 * receives the density of the second half step. */
int orc_step(const orc_problem *pb, double dz, double *Ad, double *rho)
{
    int nr = pb->nr, nt = pb->nt;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!tmp) return -3;
    for (int m = 0; m < nr; ++m)
        orc_nl_half(pb, 0.5 * dz, Ad + (size_t)2 * m * nt, tmp);
    int rc = orc_linear_step(pb, dz, Ad);
    for (int m = 0; m < nr && rc == 0; ++m)
        orc_nl_half(pb, 0.5 * dz, Ad + (size_t)2 * m * nt,
                    rho ? rho + (size_t)m * nt : tmp);
    free(tmp);
    return rc;
}

int orc_run(const orc_problem *pb, double dz, long nsteps, double *A, double *rho)
{
    for (long n = 0; n < nsteps; ++n) {
        int rc = orc_step(pb, dz, A, rho);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Multi-core timing mode: a parallel-for over rows and frequency bins  */
/* ------------------------------------------------------------------ */

/* The rows of a row phase and the bins of a column phase are independent
 * problems, so a host pool of threads can split each phase into contiguous
 * ranges (the paper's Sec. 4 runs its CPU code this way; here it only serves
 * to time the oracle on many cores).  The pool is generic: the caller hands
 * it one range task at a time and waits until every member has finished its
 * share.  Every row and bin runs exactly the per-row and per-bin functions
 * the serial step uses, so the result is bit-identical to it. */
typedef int (*orc_range_fn)(void *ctx, long i0, long i1, void *scratch);

/* Start gate: members wait until all of them exist (state 1) or one could
 * not be created (state -1, all leave), so that no member ever waits on a
 * barrier that lacks a thread. */
typedef struct {
    pthread_mutex_t mu;
    pthread_cond_t cv;
    int state;               /* 0 wait, 1 run, -1 abort */
} orc_gate;

static int orc_gate_wait(orc_gate *g)
{
    pthread_mutex_lock(&g->mu);
    while (g->state == 0) pthread_cond_wait(&g->cv, &g->mu);
    int go = g->state == 1;
    pthread_mutex_unlock(&g->mu);
    return go;
}

static void orc_gate_open(orc_gate *g, int state)
{
    pthread_mutex_lock(&g->mu);
    g->state = state;
    pthread_cond_broadcast(&g->cv);
    pthread_mutex_unlock(&g->mu);
}

typedef struct orc_pool orc_pool;
typedef struct {
    orc_pool *pool;
    int id;
    void *scratch;           /* the member's own work space */
    int rc;                  /* first nonzero status of its tasks */
} orc_member;

struct orc_pool {
    int n, started;
    pthread_t *th;
    orc_member *mem;
    pthread_barrier_t go, done;
    orc_gate gate;
    orc_range_fn fn;         /* the current parallel-for body */
    void *ctx;
    long items;
    int quit;
};

/* Member m's share of the current task: items [items m / n, items (m+1) / n). */
static void orc_pool_share(orc_pool *p, orc_member *m)
{
    long i0 = p->items * m->id / p->n, i1 = p->items * (m->id + 1) / p->n;
    if (i1 > i0) {
        int rc = p->fn(p->ctx, i0, i1, m->scratch);
        if (rc && !m->rc) m->rc = rc;
    }
}

static void *orc_pool_main(void *arg)
{
    orc_member *m = (orc_member *)arg;
    orc_pool *p = m->pool;
    if (!orc_gate_wait(&p->gate)) return NULL;
    for (;;) {
        pthread_barrier_wait(&p->go);
        if (p->quit) return NULL;
        orc_pool_share(p, m);
        pthread_barrier_wait(&p->done);
    }
}

/* Runs fn over items 0..items-1 on all members (the caller is member 0). */
static void orc_pool_run(orc_pool *p, orc_range_fn fn, void *ctx, long items)
{
    p->fn = fn;
    p->ctx = ctx;
    p->items = items;
    if (p->n > 1) pthread_barrier_wait(&p->go);
    orc_pool_share(p, &p->mem[0]);
    if (p->n > 1) pthread_barrier_wait(&p->done);
}

/* First nonzero status of any member since the pool started. */
static int orc_pool_status(const orc_pool *p)
{
    for (int k = 0; k < p->n; ++k)
        if (p->mem[k].rc) return p->mem[k].rc;
    return 0;
}

static void orc_pool_free_scratch(orc_pool *p)
{
    for (int k = 0; k < p->n; ++k) free(p->mem[k].scratch);
}

/* A pool of n members with scratch_bytes of work space each; NULL when an
 * allocation, a barrier or a thread could not be made. */
static orc_pool *orc_pool_create(int n, size_t scratch_bytes)
{
    if (n < 1) n = 1;
    orc_pool *p = (orc_pool *)calloc(1, sizeof(orc_pool));
    if (!p) return NULL;
    p->n = n;
    p->th = (pthread_t *)calloc((size_t)n, sizeof(pthread_t));
    p->mem = (orc_member *)calloc((size_t)n, sizeof(orc_member));
    int ok = p->th && p->mem;
    for (int k = 0; ok && k < n; ++k) {
        p->mem[k].pool = p;
        p->mem[k].id = k;
        p->mem[k].scratch = malloc(scratch_bytes);
        if (!p->mem[k].scratch) ok = 0;
    }
    if (!ok) {
        if (p->mem) orc_pool_free_scratch(p);
        free(p->th);
        free(p->mem);
        free(p);
        return NULL;
    }
    p->started = 1;
    if (n > 1) {
        if (pthread_barrier_init(&p->go, NULL, (unsigned)n)) ok = 0;
        if (ok && pthread_barrier_init(&p->done, NULL, (unsigned)n)) {
            pthread_barrier_destroy(&p->go);
            ok = 0;
        }
        if (!ok) {
            orc_pool_free_scratch(p);
            free(p->th);
            free(p->mem);
            free(p);
            return NULL;
        }
        pthread_mutex_init(&p->gate.mu, NULL);
        pthread_cond_init(&p->gate.cv, NULL);
        p->gate.state = 0;
        for (int k = 1; k < n; ++k) {
            if (pthread_create(&p->th[k], NULL, orc_pool_main, &p->mem[k])) break;
            ++p->started;
        }
        orc_gate_open(&p->gate, p->started == n ? 1 : -1);
        if (p->started != n) {
            for (int k = 1; k < p->started; ++k) pthread_join(p->th[k], NULL);
            pthread_barrier_destroy(&p->go);
            pthread_barrier_destroy(&p->done);
            pthread_cond_destroy(&p->gate.cv);
            pthread_mutex_destroy(&p->gate.mu);
            orc_pool_free_scratch(p);
            free(p->th);
            free(p->mem);
            free(p);
            return NULL;
        }
    }
    return p;
}

static void orc_pool_destroy(orc_pool *p)
{
    if (!p) return;
    if (p->n > 1) {
        p->quit = 1;
        pthread_barrier_wait(&p->go);
        for (int k = 1; k < p->n; ++k) pthread_join(p->th[k], NULL);
        pthread_barrier_destroy(&p->go);
        pthread_barrier_destroy(&p->done);
        pthread_cond_destroy(&p->gate.cv);
        pthread_mutex_destroy(&p->gate.mu);
    }
    orc_pool_free_scratch(p);
    free(p->th);
    free(p->mem);
    free(p);
}

/* Range tasks of one Strang step on the radial grid.  Scratch: nt doubles
 * (the density of a half step that is not kept) then 8 nr complex values
 * (cn_column's work space). */
typedef struct {
    const orc_problem *pb;
    double dz;
    cplx *A;
    double *rho;
} orc_step_ctx;

static double *scratch_rho(void *s) { return (double *)s; }

static cplx *scratch_cn(void *s, int nt) { return (cplx *)((double *)s + 2 * ((nt + 1) / 2)); }

/* Rows m0..m1-1 before the column phase: half step, then forward transform. */
static int task_rows_open(void *c, long m0, long m1, void *s)
{
    orc_step_ctx *x = (orc_step_ctx *)c;
    int nt = x->pb->nt, rc = 0;
    for (long m = m0; m < m1; ++m) {
        double *row = (double *)(x->A + (size_t)m * nt);
        orc_nl_half(x->pb, 0.5 * x->dz, row, scratch_rho(s));
        if (orc_fft(row, nt, 0)) rc = -1;
    }
    return rc;
}

/* Frequency bins q0..q1-1: one tridiagonal solve each. */
static int task_columns(void *c, long q0, long q1, void *s)
{
    orc_step_ctx *x = (orc_step_ctx *)c;
    int rc = 0;
    for (long q = q0; q < q1; ++q)
        if (cn_column(x->pb, x->dz, x->A, (int)q, scratch_cn(s, x->pb->nt))) rc = -2;
    return rc;
}

/* Rows m0..m1-1 after the column phase: inverse transform, then half step. */
static int task_rows_close(void *c, long m0, long m1, void *s)
{
    orc_step_ctx *x = (orc_step_ctx *)c;
    int nt = x->pb->nt, rc = 0;
    for (long m = m0; m < m1; ++m) {
        double *row = (double *)(x->A + (size_t)m * nt);
        if (orc_fft(row, nt, 1)) rc = -1;
        orc_nl_half(x->pb, 0.5 * x->dz, row, x->rho ? x->rho + (size_t)m * nt : scratch_rho(s));
    }
    return rc;
}

int orc_run_threads(const orc_problem *pb, double dz, long nsteps, double *A, double *rho, int nthreads)
{
    int nt = pb->nt, nr = pb->nr;
    size_t bytes = sizeof(double) * 2 * (size_t)((nt + 1) / 2) + sizeof(cplx) * 8 * (size_t)nr;
    orc_pool *p = orc_pool_create(nthreads, bytes);
    if (!p) return -3;
    orc_step_ctx x = {pb, dz, (cplx *)A, rho};
    for (long n = 0; n < nsteps && !orc_pool_status(p); ++n) {
        orc_pool_run(p, task_rows_open, &x, nr);
        orc_pool_run(p, task_columns, &x, nt);
        orc_pool_run(p, task_rows_close, &x, nr);
    }
    int rc = orc_pool_status(p);
    orc_pool_destroy(p);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics (quantities of Fig. 4 plus energy, peaks, spectrum)     */
/* ------------------------------------------------------------------ */

/* Radial weight of row m in the area integral 2 pi int r dr:
 * 2 pi dr^2 W_m with W_0 = 1/8 (disc of radius dr/2) and W_m = m.  These are
 * also the weights in which the Crank-Nicolson operator is self-adjoint. */
static double radial_weight(int m) { return m == 0 ? 0.125 : (double)m; }

/* energy = 2 pi dr^2 dtau sum_m W_m sum_p |A_mp|^2;
 * power[p] = 2 pi dr^2 sum_m W_m |A_mp|^2 (nt values, nullable);
 * fluence[m] = dtau sum_p |A_mp|^2 (nr values, nullable);
 * spectral_rms from S_q = sum_m W_m |FFT(A_m.)_q|^2. */
void orc_diag_compute(const orc_problem *pb, const double *Ad, const double *rho,
                      orc_diag *out, double *power, double *fluence)
{
    int nr = pb->nr, nt = pb->nt;
    const cplx *A = (const cplx *)Ad;
    double dr = pb->r_max / (double)(nr - 1);
    double dtau = pb->t_window / nt;
    double area = 2.0 * ORC_PI * dr * dr;
    memset(out, 0, sizeof(*out));
    if (power) for (int p = 0; p < nt; ++p) power[p] = 0.0;
    double esum = 0.0;
    for (int m = 0; m < nr; ++m) {
        double rowsum = 0.0;
        for (int p = 0; p < nt; ++p) {
            cplx v = A[(size_t)m * nt + p];
            double re = creal(v), im = cimag(v);
            if (!isfinite(re) || !isfinite(im)) out->nonfinite = 1;
            double i2 = re * re + im * im;
            rowsum += i2;
            if (i2 > out->peak_intensity) out->peak_intensity = i2;
            if (m == 0 && i2 > out->onaxis_peak) out->onaxis_peak = i2;
            if (power) power[p] += area * radial_weight(m) * i2;
        }
        esum += radial_weight(m) * rowsum;
        if (fluence) fluence[m] = dtau * rowsum;
    }
    out->energy = area * dtau * esum;
    if (rho) {
        for (size_t i = 0; i < (size_t)nr * nt; ++i)
            if (rho[i] > out->peak_rho) out->peak_rho = rho[i];
    }
    /* spectral rms width (no memory: NaN) */
    double *row = (double *)malloc(sizeof(double) * 2 * (size_t)nt);
    if (!row) { out->spectral_rms = NAN; return; }
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int m = 0; m < nr; ++m) {
        memcpy(row, A + (size_t)m * nt, sizeof(double) * 2 * (size_t)nt);
        orc_fft(row, nt, 0);
        for (int q = 0; q < nt; ++q) {
            double sq = radial_weight(m) * (row[2 * q] * row[2 * q] + row[2 * q + 1] * row[2 * q + 1]);
            double w = orc_omega(pb, q);
            s0 += sq;
            s1 += sq * w;
            s2 += sq * w * w;
        }
    }
    free(row);
    if (s0 > 0) {
        double mean = s1 / s0;
        double var = s2 / s0 - mean * mean;
        out->spectral_rms = var > 0 ? sqrt(var) : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Cartesian transverse grid (reading R9)                              */
/* ------------------------------------------------------------------ */

/* Line of n nodes, spacing h, walls at nodes 0 and n-1.  With
 * s = dz/(4 k0 h^2) (Eqs. (diff1)-(diff2) on one axis) and
 * delta_q = k'' omega_q^2 dz/4 when with_disp:
 *   rows 0, n-1 : b = 1, a = c = d = e = f = 0               (A = 0)
 *   1..n-2      : a = c = -is, b = 1 + 2is - i delta
 *                 d = f =  is, e = 1 - 2is + i delta          */
void orc_xy_cn_coeffs(const orc_problem *pb, double dz, int q, int n, double h, int with_disp,
                      double *ad, double *bd, double *cd, double *dd, double *ed, double *fd)
{
    cplx *a = (cplx *)ad, *b = (cplx *)bd, *c = (cplx *)cd;
    cplx *d = (cplx *)dd, *e = (cplx *)ed, *f = (cplx *)fd;
    double k0 = orc_k0(pb);
    double s = (pb->flags & ORC_DIFFRACTION) ? dz / (4.0 * k0 * h * h) : 0.0;
    double w = orc_omega(pb, q);
    double delta = (with_disp && (pb->flags & ORC_DISPERSION) && !(pb->flags & ORC_EXACT_DISPERSION))
                       ? pb->k2 * w * w * dz / 4.0 : 0.0;
    for (int j = 0; j < n; ++j) {
        if (j == 0 || j == n - 1) {
            a[j] = 0; b[j] = 1.0; c[j] = 0; d[j] = 0; e[j] = 0; f[j] = 0;
        } else {
            a[j] = -I * s;
            b[j] = 1.0 + I * (2.0 * s) - I * delta;
            c[j] = -I * s;
            d[j] = I * s;
            e[j] = 1.0 - I * (2.0 * s) + I * delta;
            f[j] = I * s;
        }
    }
}

/* One transverse line of bin q: the n values at A[off + k stride],
 * k = 0..n-1, replaced by (M_abc)^-1 M_def times them (and, in the y factor
 * under ORC_EXACT_DISPERSION, by the exact dispersion factor).
 * co: scratch of 8 n complex values. */
static int xy_line(const orc_problem *pb, double dz, int q, int n, double h, int with_disp,
                   cplx *A, size_t off, size_t stride, cplx *co)
{
    cplx *a = co, *b = co + n, *c = co + 2 * n, *d = co + 3 * n;
    cplx *e = co + 4 * n, *f = co + 5 * n, *col = co + 6 * n, *rhs = co + 7 * n;
    orc_xy_cn_coeffs(pb, dz, q, n, h, with_disp, (double *)a, (double *)b, (double *)c,
                     (double *)d, (double *)e, (double *)f);
    for (int k = 0; k < n; ++k) col[k] = A[off + (size_t)k * stride];
    for (int k = 0; k < n; ++k) {
        cplx v = e[k] * col[k];
        if (k > 0) v += d[k] * col[k - 1];
        if (k < n - 1) v += f[k] * col[k + 1];
        rhs[k] = v;
    }
    int rc = orc_thomas(n, (double *)a, (double *)b, (double *)c, (double *)rhs, (double *)col);
    cplx ph = 1.0;
    if (with_disp && (pb->flags & ORC_DISPERSION) && (pb->flags & ORC_EXACT_DISPERSION)) {
        double w = orc_omega(pb, q);
        ph = cexp(I * (pb->k2 * w * w * dz / 2.0));
    }
    for (int k = 0; k < n; ++k) A[off + (size_t)k * stride] = ph * col[k];
    return rc;
}

/* A <- F^-1( C_y C_x F(A) ): transform every (x, y) row along tau, then per
 * frequency bin the x factor on every x line and the y factor on every y
 * line, then the inverse transform. */
int orc_xy_linear_step(const orc_problem *pb, const orc_xy_grid *g, double dz, double *Ad)
{
    int nx = g->nx, ny = g->ny, nt = pb->nt;
    double dx = g->x_width / (double)(nx - 1), dy = g->y_width / (double)(ny - 1);
    size_t rows = (size_t)nx * ny;
    cplx *A = (cplx *)Ad;
    for (size_t m = 0; m < rows; ++m)
        if (orc_fft((double *)(A + m * nt), nt, 0)) return -1;
    int nmax = nx > ny ? nx : ny;
    cplx *co = (cplx *)malloc(sizeof(cplx) * (size_t)nmax * 8);
    if (!co) return -3;
    int rc = 0;
    for (int q = 0; q < nt && rc == 0; ++q) {
        /* x factor: line (j, q) holds A[i][j][q], i = 0..nx-1 */
        for (int j = 0; j < ny && rc == 0; ++j)
            rc = xy_line(pb, dz, q, nx, dx, 0, A, (size_t)j * nt + q, (size_t)ny * nt, co);
        /* y factor with the dispersion term: line (i, q) holds A[i][j][q] */
        for (int i = 0; i < nx && rc == 0; ++i)
            rc = xy_line(pb, dz, q, ny, dy, 1, A, (size_t)i * ny * nt + q, (size_t)nt, co);
    }
    free(co);
    if (rc) return -2;
    for (size_t m = 0; m < rows; ++m)
        if (orc_fft((double *)(A + m * nt), nt, 1)) return -1;
    return 0;
}

/* One Strang step (Eq. (nlseq)) on the Cartesian grid: the nonlinear half
 * steps act on each (x, y) row exactly as on a radial row. */
int orc_xy_step(const orc_problem *pb, const orc_xy_grid *g, double dz, double *Ad, double *rho)
{
    int nt = pb->nt;
    size_t rows = (size_t)g->nx * g->ny;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nt);
    if (!tmp) return -3;
    for (size_t m = 0; m < rows; ++m) orc_nl_half(pb, 0.5 * dz, Ad + 2 * m * nt, tmp);
    int rc = orc_xy_linear_step(pb, g, dz, Ad);
    for (size_t m = 0; m < rows && rc == 0; ++m)
        orc_nl_half(pb, 0.5 * dz, Ad + 2 * m * nt, rho ? rho + m * nt : tmp);
    free(tmp);
    return rc;
}

int orc_xy_run(const orc_problem *pb, const orc_xy_grid *g, double dz, long nsteps, double *A,
               double *rho)
{
    for (long n = 0; n < nsteps; ++n) {
        int rc = orc_xy_step(pb, g, dz, A, rho);
        if (rc) return rc;
    }
    return 0;
}

/* orc_xy_run on the host pool: rows as for the radial grid, and per
 * frequency bin both factors (its x lines, then its y lines), the same
 * functions in the same order as orc_xy_step, so the result is
 * bit-identical.  Scratch: nt doubles then 8 max(nx, ny) complex values. */
typedef struct {
    const orc_problem *pb;
    const orc_xy_grid *g;
    double dz;
    cplx *A;
    double *rho;
} orc_xy_ctx;

static int task_xy_rows_open(void *c, long m0, long m1, void *s)
{
    orc_xy_ctx *x = (orc_xy_ctx *)c;
    orc_step_ctx r = {x->pb, x->dz, x->A, NULL};
    return task_rows_open(&r, m0, m1, s);
}

static int task_xy_bins(void *c, long q0, long q1, void *s)
{
    orc_xy_ctx *x = (orc_xy_ctx *)c;
    const orc_xy_grid *g = x->g;
    int nx = g->nx, ny = g->ny, nt = x->pb->nt, rc = 0;
    double dx = g->x_width / (double)(nx - 1), dy = g->y_width / (double)(ny - 1);
    cplx *co = scratch_cn(s, nt);
    for (long q = q0; q < q1; ++q) {
        for (int j = 0; j < ny; ++j)
            if (xy_line(x->pb, x->dz, (int)q, nx, dx, 0, x->A, (size_t)j * nt + q, (size_t)ny * nt, co))
                rc = -2;
        for (int i = 0; i < nx; ++i)
            if (xy_line(x->pb, x->dz, (int)q, ny, dy, 1, x->A, (size_t)i * ny * nt + q, (size_t)nt, co))
                rc = -2;
    }
    return rc;
}

static int task_xy_rows_close(void *c, long m0, long m1, void *s)
{
    orc_xy_ctx *x = (orc_xy_ctx *)c;
    orc_step_ctx r = {x->pb, x->dz, x->A, x->rho};
    return task_rows_close(&r, m0, m1, s);
}

int orc_xy_run_threads(const orc_problem *pb, const orc_xy_grid *g, double dz, long nsteps, double *A,
                       double *rho, int nthreads)
{
    int nt = pb->nt, nmax = g->nx > g->ny ? g->nx : g->ny;
    long rows = (long)g->nx * g->ny;
    size_t bytes = sizeof(double) * 2 * (size_t)((nt + 1) / 2) + sizeof(cplx) * 8 * (size_t)nmax;
    orc_pool *p = orc_pool_create(nthreads, bytes);
    if (!p) return -3;
    orc_xy_ctx x = {pb, g, dz, (cplx *)A, rho};
    for (long n = 0; n < nsteps && !orc_pool_status(p); ++n) {
        orc_pool_run(p, task_xy_rows_open, &x, rows);
        orc_pool_run(p, task_xy_bins, &x, nt);
        orc_pool_run(p, task_xy_rows_close, &x, rows);
    }
    int rc = orc_pool_status(p);
    orc_pool_destroy(p);
    return rc;
}

void orc_xy_diag(const orc_problem *pb, const orc_xy_grid *g, const double *Ad, const double *rho,
                 orc_diag *out)
{
    int nx = g->nx, ny = g->ny, nt = pb->nt;
    size_t rows = (size_t)nx * ny;
    size_t centre = (size_t)((nx - 1) / 2) * ny + (size_t)((ny - 1) / 2);
    double dx = g->x_width / (double)(nx - 1), dy = g->y_width / (double)(ny - 1);
    double dtau = pb->t_window / nt;
    const cplx *A = (const cplx *)Ad;
    memset(out, 0, sizeof(*out));
    double esum = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    double *row = (double *)malloc(sizeof(double) * 2 * (size_t)nt);
    if (!row) {                      /* no memory: every diagnostic NaN */
        out->energy = out->peak_intensity = out->onaxis_peak = out->peak_rho = out->spectral_rms = NAN;
        out->nonfinite = 1;
        return;
    }
    for (size_t m = 0; m < rows; ++m) {
        for (int p = 0; p < nt; ++p) {
            cplx v = A[m * nt + p];
            double re = creal(v), im = cimag(v);
            if (!isfinite(re) || !isfinite(im)) out->nonfinite = 1;
            double i2 = re * re + im * im;
            esum += i2;
            if (i2 > out->peak_intensity) out->peak_intensity = i2;
            if (m == centre && i2 > out->onaxis_peak) out->onaxis_peak = i2;
        }
        memcpy(row, A + m * nt, sizeof(double) * 2 * (size_t)nt);
        orc_fft(row, nt, 0);
        for (int q = 0; q < nt; ++q) {
            double sq = row[2 * q] * row[2 * q] + row[2 * q + 1] * row[2 * q + 1];
            double w = orc_omega(pb, q);
            s0 += sq;
            s1 += sq * w;
            s2 += sq * w * w;
        }
    }
    free(row);
    out->energy = dx * dy * dtau * esum;
    if (rho)
        for (size_t i = 0; i < rows * nt; ++i)
            if (rho[i] > out->peak_rho) out->peak_rho = rho[i];
    if (s0 > 0) {
        double mean = s1 / s0;
        double var = s2 / s0 - mean * mean;
        out->spectral_rms = var > 0 ? sqrt(var) : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Step-doubling dz controller (not in the paper: it uses a fixed dz)  */
/* ------------------------------------------------------------------ */

static double rel_l2(size_t n2, const double *x, const double *ref)
{
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < n2; ++i) {
        double d = x[i] - ref[i];
        num += d * d;
        den += ref[i] * ref[i];
    }
    return den > 0 ? sqrt(num / den) : sqrt(num);
}

/* From state A at z0, one step of dz gives A1 and two steps of dz/2 give A2;
 * err = ||A2 - A1|| / ||A2||.  err <= rtol accepts A2.  Either way the next
 * dz is dz * clamp(0.9 (rtol/err)^(1/3), 0.2, 2) (the Strang local error is
 * O(dz^3)); err = 0 gives the factor 2.  The last step is clipped to land on
 * z_end exactly.  Fails (status -1) if dz falls below dz_min or max_reject
 * consecutive rejections occur. */
int orc_propagate_adaptive(const orc_problem *pb, double *A, double *rho,
                           double z0, double z_end, double dz0, double rtol,
                           double dz_min, int max_reject,
                           orc_adaptive_result *res)
{
    size_t n2 = (size_t)2 * pb->nr * pb->nt;
    size_t n1 = (size_t)pb->nr * pb->nt;
    double *a1 = (double *)malloc(sizeof(double) * n2);
    double *a2 = (double *)malloc(sizeof(double) * n2);
    double *r2 = (double *)malloc(sizeof(double) * n1);
    memset(res, 0, sizeof(*res));
    if (!a1 || !a2 || !r2) {
        free(a1); free(a2); free(r2);
        res->status = -3;
        return -3;
    }
    double z = z0, dz = dz0;
    int consecutive = 0;
    int status = 0;
    while (z < z_end) {
        double h = dz;
        int last = 0;
        if (z + h >= z_end) { h = z_end - z; last = 1; }
        memcpy(a1, A, sizeof(double) * n2);
        memcpy(a2, A, sizeof(double) * n2);
        orc_step(pb, h, a1, NULL);
        orc_step(pb, 0.5 * h, a2, NULL);
        orc_step(pb, 0.5 * h, a2, r2);
        double err = rel_l2(n2, a1, a2);
        res->last_err = err;
        double fac = (err > 0) ? 0.9 * cbrt(rtol / err) : 2.0;
        if (fac < 0.2) fac = 0.2;
        if (fac > 2.0) fac = 2.0;
        if (err <= rtol) {
            memcpy(A, a2, sizeof(double) * n2);
            if (rho) memcpy(rho, r2, sizeof(double) * n1);
            z = last ? z_end : z + h;
            res->accepted++;
            consecutive = 0;
            /* a clipped last step does not shrink the proposal */
            dz = last ? dz : h * fac;
        } else {
            res->rejected++;
            consecutive++;
            dz = h * fac;
        }
        if (dz < dz_min || consecutive > max_reject) { status = -1; break; }
    }
    res->z = z;
    res->dz_next = dz;
    res->status = status;
    free(a1);
    free(a2);
    free(r2);
    return status;
}

/* ------------------------------------------------------------------ */
/* Learned-dz MLP, FP64 (not in the paper)                             */
/* ------------------------------------------------------------------ */
/* Parameter layout (flat): W1[nh][nin], b1[nh], W2[nh][nh], b2[nh],
 * W3[nh], b3.  Hidden layers use tanh, the output is linear.  Loss is the
 * mean over the batch of (y - target)^2. */

static void mlp_offsets(int nin, int nh, size_t off[6])
{
    off[0] = 0;
    off[1] = off[0] + (size_t)nh * nin;
    off[2] = off[1] + (size_t)nh;
    off[3] = off[2] + (size_t)nh * nh;
    off[4] = off[3] + (size_t)nh;
    off[5] = off[4] + (size_t)nh;
}

int orc_mlp_forward(int batch, int nin, int nh, const double *pr,
                    const double *x, double *y)
{
    size_t o[6];
    mlp_offsets(nin, nh, o);
    double *h1 = (double *)malloc(sizeof(double) * (size_t)nh);
    double *h2 = (double *)malloc(sizeof(double) * (size_t)nh);
    if (!h1 || !h2) { free(h1); free(h2); return -3; }
    for (int b = 0; b < batch; ++b) {
        const double *xb = x + (size_t)b * nin;
        for (int i = 0; i < nh; ++i) {
            double s = pr[o[1] + i];
            for (int k = 0; k < nin; ++k) s += pr[o[0] + (size_t)i * nin + k] * xb[k];
            h1[i] = tanh(s);
        }
        for (int i = 0; i < nh; ++i) {
            double s = pr[o[3] + i];
            for (int k = 0; k < nh; ++k) s += pr[o[2] + (size_t)i * nh + k] * h1[k];
            h2[i] = tanh(s);
        }
        double s = pr[o[5]];
        for (int k = 0; k < nh; ++k) s += pr[o[4] + k] * h2[k];
        y[b] = s;
    }
    free(h1);
    free(h2);
    return 0;
}

/* Loss and its gradient by reverse-mode differentiation of the forward pass
 * above (chain rule layer by layer; tanh' = 1 - tanh^2). */
int orc_mlp_loss_grad(int batch, int nin, int nh, const double *pr,
                      const double *x, const double *target,
                      double *loss, double *grad)
{
    size_t o[6];
    mlp_offsets(nin, nh, o);
    size_t np = o[5] + 1;
    for (size_t i = 0; i < np; ++i) grad[i] = 0.0;
    double *h1 = (double *)malloc(sizeof(double) * (size_t)nh);
    double *h2 = (double *)malloc(sizeof(double) * (size_t)nh);
    double *g1 = (double *)malloc(sizeof(double) * (size_t)nh);
    double *g2 = (double *)malloc(sizeof(double) * (size_t)nh);
    if (!h1 || !h2 || !g1 || !g2) { free(h1); free(h2); free(g1); free(g2); return -3; }
    double total = 0.0;
    for (int b = 0; b < batch; ++b) {
        const double *xb = x + (size_t)b * nin;
        for (int i = 0; i < nh; ++i) {
            double s = pr[o[1] + i];
            for (int k = 0; k < nin; ++k) s += pr[o[0] + (size_t)i * nin + k] * xb[k];
            h1[i] = tanh(s);
        }
        for (int i = 0; i < nh; ++i) {
            double s = pr[o[3] + i];
            for (int k = 0; k < nh; ++k) s += pr[o[2] + (size_t)i * nh + k] * h1[k];
            h2[i] = tanh(s);
        }
        double y = pr[o[5]];
        for (int k = 0; k < nh; ++k) y += pr[o[4] + k] * h2[k];
        double r = y - target[b];
        total += r * r;
        double gy = 2.0 * r / batch;            /* d loss / d y */
        grad[o[5]] += gy;
        for (int k = 0; k < nh; ++k) {
            grad[o[4] + k] += gy * h2[k];
            g2[k] = gy * pr[o[4] + k] * (1.0 - h2[k] * h2[k]);   /* d/d pre2 */
        }
        for (int i = 0; i < nh; ++i) {
            grad[o[3] + i] += g2[i];
            for (int k = 0; k < nh; ++k) grad[o[2] + (size_t)i * nh + k] += g2[i] * h1[k];
        }
        for (int k = 0; k < nh; ++k) {
            double s = 0.0;
            for (int i = 0; i < nh; ++i) s += pr[o[2] + (size_t)i * nh + k] * g2[i];
            g1[k] = s * (1.0 - h1[k] * h1[k]);                   /* d/d pre1 */
        }
        for (int i = 0; i < nh; ++i) {
            grad[o[1] + i] += g1[i];
            for (int k = 0; k < nin; ++k) grad[o[0] + (size_t)i * nin + k] += g1[i] * xb[k];
        }
    }
    *loss = total / batch;
    free(h1);
    free(h2);
    free(g1);
    free(g2);
    return 0;
}
