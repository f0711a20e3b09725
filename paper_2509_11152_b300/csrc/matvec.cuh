// H^2 matvec and refinement vector kernels (float64).
#pragma once

#include "h2rs_internal.h"

namespace h2rs {

// y = A x on the device.  The coefficient vectors (2 * sum(rank) * nrhs doubles) are
// allocated stream-ordered, or taken from `scratch` when it is not null.
void matvec_dev(const MatrixObj& M, int nrhs, const double* x, int64_t ldx, double* y, int64_t ldy,
                cudaStream_t s, double* scratch = nullptr);

// r = b - y;  x += d;  out[c] = ||v_c||^2  (all n x nrhs column-major, device)
void residual_dev(const double* b, int64_t ldb, const double* y, int64_t ldy, double* r, int64_t ldr,
                  int64_t n, int nrhs, cudaStream_t s);
void add_dev(double* x, int64_t ldx, const double* d, int64_t ldd, int64_t n, int nrhs, cudaStream_t s);
void colnorm2_dev(const double* v, int64_t ldv, int64_t n, int nrhs, double* out, cudaStream_t s);
// out[c * nseg + z] = squared norm of rows seg[z] .. seg[z+1]-1 of column c (seg: device)
void segnorm2_dev(const double* v, int64_t ldv, const int64_t* seg, int nseg, int nrhs, double* out,
                  cudaStream_t s);

// GMRES helpers on n x nrhs column blocks stored contiguously (ld n):
// h[i*nrhs+c] = <V_i[:,c], w[:,c]>;  w[:,c] += sum_i coef[i*nrhs+c] V_i[:,c];  y = diag(sc) x
void multidot_dev(const double* V, const double* w, int m, int64_t n, int nrhs, double* h, cudaStream_t s);
void combine_dev(const double* V, const double* coef, int m, int64_t n, int nrhs, double* w, cudaStream_t s);
void scale_dev(const double* x, const double* sc, int64_t n, int nrhs, double* y, cudaStream_t s);

}  // namespace h2rs
