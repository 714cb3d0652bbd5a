// fcn_host.h -- host helpers of fcn_api.cu used by the Cartesian-grid API
// (xy_api.cu): argument checks, nonlinear-step coefficients, the FFT
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
cudaError_t twiddles(int nt, const cx<T> **out);
// k0 = 2 pi n0/lambda0, dtau = T/Nt, domega = 2 pi/(Nt dtau).
void consts(const fcn_grid &g, const fcn_params &p, double *k0, double *dtau, double *domega);
}  // namespace hostx
}  // namespace fcn
