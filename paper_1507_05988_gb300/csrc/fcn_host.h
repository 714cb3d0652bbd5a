// fcn_host.h -- host helpers of fcn_api.cu used by the Cartesian-grid API
// (xy_api.cu) and the allocation-free column stage (noalloc.cu): argument
// checks, Crank-Nicolson coefficients, nonlinear-step coefficients, the FFT
// twiddle tables and the derived constants of one grid and parameter set.
#pragma once

#include <string>

#include "../../include/fcn.h"
#include "fcn_device.cuh"

namespace fcn {
namespace hostx {
// Checks grid (nr, nt, r_max, t_window), precision and physics parameters.
int check_params(int prec, const fcn_grid *g, const fcn_params *p, std::string *why);
// Coefficients of a nonlinear half step of length h (Eq. (nonlinearpart)).
template <typename T>
NLCoef<T> nl(const fcn_grid &g, const fcn_params &p, double h);
// Process-wide twiddle table of the row stage's FFT of nt points.
template <typename T>
cudaError_t twiddles(int ntp, const cx<T> **out);   // ntp: Nt with the FFT plan tag (fft_tag)
// k0 = 2 pi n0/lambda0, dtau = T/Nt, domega = 2 pi/(Nt dtau).
void consts(const fcn_grid &g, const fcn_params &p, double *k0, double *dtau, double *domega);
// s = dz/(4 k0 dr^2) and dk (delta_q = dk q^2) of the Crank-Nicolson system;
// with FCN_EXACT_DISPERSION dk = 0 and *disp receives the coefficient of the
// exact factor exp(2 i disp q^2) applied instead (disp may be NULL).
void cn_coefs(const fcn_grid &g, const fcn_params &p, double dz, double *s, double *dk,
              double *disp);
}  // namespace hostx
}  // namespace fcn
