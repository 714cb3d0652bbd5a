/*
 * fcn_oracle.h -- plain FP64 CPU oracle of the split-step Fourier /
 * Crank-Nicolson (FCN) z-step of Ma & Lin, "Parallel simulation for the
 * ultra-short laser pulses' propagation in air" (arXiv:1507.05988).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Units are SI throughout.  Complex arrays are interleaved (re, im) doubles.
 * The field is stored row-major as A[m][p]: m = radial index (m = 0 is the
 * axis), p = time index (contiguous).
 *
 * Parity status per function (see the matching tests):
 *   orc_fft, orc_thomas, orc_cn_coeffs, orc_rho_row, orc_nl_half,
 *   orc_linear_step, orc_step, orc_diag : pinned (closed forms, invariants,
 *     brute force, library routines).
 *   orc_propagate_adaptive : pinned (controller arithmetic and exact
 *     landing on z_end; the step it wraps is pinned above).
 *   orc_mlp_* : pinned (finite differences, closed-form tiny nets).
 *   orc_xy_* (Cartesian transverse grid) : pinned (elliptical Gaussian beam
 *     in closed form, dense solves of the 1-D systems, energy, the discrete
 *     dispersion factor, pure SPM, agreement with the radial solver, the
 *     unsplit 2-D step at third order; the threaded run bit-identical).
 *   Full coupled run (all physics on) : parity unpinned beyond the
 *     invariants above -- the paper prints no values for it.
 */
#ifndef FCN_ORACLE_H
#define FCN_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Physics switches (bit flags). */
#define ORC_DIFFRACTION   1u   /* (i/2k0) Delta_perp term of Eq. (linearpart)   */
#define ORC_DISPERSION    2u   /* -(i k''/2) d^2/dt^2 term of Eq. (linearpart)  */
#define ORC_KERR          4u   /* sum_j n_2j |A|^2j term of Eq. (nonlinearpart) */
#define ORC_PLASMA        8u   /* plasma defocusing term of Eq. (nonlinearpart) */
#define ORC_MPI          16u   /* multiphoton loss term of Eq. (nonlinearpart)  */
#define ORC_MPI_SAT      32u   /* optional (1 - rho/rho_nt) factor on the loss  */
#define ORC_PRINTED_CJ   64u   /* use c_j, f_j exactly as printed in Sec. 3
                                  (factor 1 - 1/(2j)); only for demonstrating
                                  that the pins reject that reading          */
#define ORC_EXACT_DISPERSION 128u /* variant of reading R7: the CN system for
                                  diffraction alone, then each frequency
                                  column times its exact dispersion factor
                                  exp(i k'' omega_q^2 dz / 2) (the two linear
                                  operators act on r and on omega and commute) */

typedef struct {
    int    nr;          /* radial points, >= 3; dr = r_max / (nr - 1)      */
    int    nt;          /* time points, power of two; dtau = t_window / nt  */
    double r_max;       /* m                                                */
    double t_window;    /* s; tau_p = -t_window/2 + p * dtau                */
    double lambda0;     /* m                                                */
    double n0;          /* linear index                                     */
    double n2j[4];      /* n2 [m^2/W], n4 [m^4/W^2], n6, n8                 */
    double k2;          /* GVD k'' [s^2/m]                                  */
    double sigma_k;     /* MPI cross section [s^-1 m^(2K) W^-K]             */
    double rho_nt;      /* neutral density [m^-3]                           */
    int    K;           /* photon number                                    */
    unsigned flags;     /* ORC_* bits                                       */
} orc_problem;

typedef struct {
    double energy;        /* J: 2 pi dr^2 dtau sum_m W_m sum_p |A|^2        */
    double peak_intensity;/* W/m^2                                          */
    double peak_rho;      /* m^-3 (of the supplied rho array)               */
    double onaxis_peak;   /* W/m^2: max_p |A_{0,p}|^2                        */
    double spectral_rms;  /* rad/s: rms width of omega, energy-weighted      */
    int    nonfinite;     /* 1 if any field entry is NaN/Inf                 */
} orc_diag;

typedef struct {
    double z;             /* position reached                              */
    double dz_next;       /* proposal for the next step                    */
    long   accepted;
    long   rejected;
    double last_err;
    int    status;        /* 0 ok, -1 dz underflow / too many rejections, */
                          /* -3 no memory                                   */
} orc_adaptive_result;

/* Derived constants. */
double orc_k0(const orc_problem *pb);
double orc_omega0(const orc_problem *pb);
double orc_rho_c(const orc_problem *pb);
double orc_beta_k(const orc_problem *pb);
double orc_omega(const orc_problem *pb, int q);

/* Building blocks. */
int  orc_fft(double *x, int n, int inverse);
int  orc_thomas(int n, const double *a, const double *b, const double *c,
                const double *d, double *x);
void orc_cn_coeffs(const orc_problem *pb, double dz, int q,
                   double *a, double *b, double *c,
                   double *d, double *e, double *f);
void orc_rho_row(const orc_problem *pb, const double *intensity, double *rho);
void orc_nl_half(const orc_problem *pb, double h, double *row, double *rho);

/* Whole steps. */
int  orc_linear_step(const orc_problem *pb, double dz, double *A);
int  orc_step(const orc_problem *pb, double dz, double *A, double *rho);
int  orc_run(const orc_problem *pb, double dz, long nsteps, double *A, double *rho);
/* orc_run with the paper's row/column thread decomposition (Sec. 4);
 * bit-identical results; for timing on multi-core hosts. */
int  orc_run_threads(const orc_problem *pb, double dz, long nsteps, double *A, double *rho,
                     int nthreads);
void orc_diag_compute(const orc_problem *pb, const double *A, const double *rho,
                      orc_diag *out, double *power, double *fluence);
int  orc_propagate_adaptive(const orc_problem *pb, double *A, double *rho,
                            double z0, double z_end, double dz0, double rtol,
                            double dz_min, int max_reject,
                            orc_adaptive_result *res);

/* Cartesian transverse grid (Sec. 2: Delta_perp = d^2/dx^2 + d^2/dy^2 for
 * beams without cylindrical symmetry).  The physics and the time grid come
 * from an orc_problem (nr and r_max unused); the field is A[i][j][p] with
 * x_i = -x_width/2 + i dx, dx = x_width/(nx - 1), likewise y_j, and A = 0 on
 * the four walls i = 0, nx-1, j = 0, ny-1.  The linear step is the product
 * of the Crank-Nicolson (Cayley) factors of the x and the y part (reading
 * R9 in fcn_oracle.c). */
typedef struct {
    int    nx, ny;      /* >= 3 */
    double x_width;     /* m */
    double y_width;     /* m */
} orc_xy_grid;

/* Diagonals of the Crank-Nicolson system of one transverse line of n nodes
 * with spacing h (nodes 0 and n-1 are the walls); with_disp = 1 puts the
 * dispersion term of bin q into it. */
void orc_xy_cn_coeffs(const orc_problem *pb, double dz, int q, int n, double h, int with_disp,
                      double *a, double *b, double *c, double *d, double *e, double *f);
int  orc_xy_linear_step(const orc_problem *pb, const orc_xy_grid *g, double dz, double *A);
int  orc_xy_step(const orc_problem *pb, const orc_xy_grid *g, double dz, double *A, double *rho);
int  orc_xy_run(const orc_problem *pb, const orc_xy_grid *g, double dz, long nsteps, double *A,
                double *rho);
/* orc_xy_run with rows and frequency bins split over nthreads threads
 * (Sec. 4's decomposition); bit-identical results; for timing. */
int  orc_xy_run_threads(const orc_problem *pb, const orc_xy_grid *g, double dz, long nsteps,
                        double *A, double *rho, int nthreads);
/* energy = dx dy dtau sum |A|^2; onaxis_peak on the row nearest the centre
 * (i = (nx-1)/2, j = (ny-1)/2); spectral_rms from the unweighted spectrum. */
void orc_xy_diag(const orc_problem *pb, const orc_xy_grid *g, const double *A, const double *rho,
                 orc_diag *out);

/* Learned-dz MLP (6 -> H -> H -> 1, tanh hidden, linear output), FP64. */
int  orc_mlp_forward(int batch, int nin, int nh, const double *params,
                     const double *x, double *y);
int  orc_mlp_loss_grad(int batch, int nin, int nh, const double *params,
                       const double *x, const double *target,
                       double *loss, double *grad);

#ifdef __cplusplus
}
#endif
#endif
