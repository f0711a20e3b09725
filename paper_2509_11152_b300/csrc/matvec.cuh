// H^2 matvec and refinement vector kernels (float64).
#pragma once

#include "h2rs_internal.h"

namespace h2rs {

// y = A x on the device.  The coefficient vectors (2 * sum(rank) * nrhs doubles) are
// allocated stream-ordered, or taken from `scratch` when it is not null.
void matvec_dev(const MatrixObj& M, int nrhs, const double* x, int64_t ldx, double* y, int64_t ldy,
                cudaStream_t s, double* scratch = nullptr);

// r = b - y;  x += d  (all n x nrhs column-major, device)
void residual_dev(const double* b, int64_t ldb, const double* y, int64_t ldy, double* r, int64_t ldr,
                  int64_t n, int nrhs, cudaStream_t s);
void add_dev(double* x, int64_t ldx, const double* d, int64_t ldd, int64_t n, int nrhs, cudaStream_t s);
// out[c * nseg + z] = squared norm of rows seg[z] .. seg[z+1]-1 of column c (seg: device)
void segnorm2_dev(const double* v, int64_t ldv, const int64_t* seg, int nseg, int nrhs, double* out,
                  cudaStream_t s);

// GMRES helpers on n x nrhs column blocks stored contiguously (ld n), per channel
// q = c * nseg + z (column c restricted to the rows seg[z] .. seg[z+1]-1 of system z;
// seg: device array of nseg+1 offsets), nq = nrhs * nseg:
// h[i*nq+q] = <V_i, w>_q;  w += sum_i coef[i*nq+q] V_i on channel q;  y = sc[q] x on q
void multidot_dev(const double* V, const double* w, int m, int64_t n, int nrhs, const int64_t* seg, int nseg,
                  double* h, cudaStream_t s);
void combine_dev(const double* V, const double* coef, int m, int64_t n, int nrhs, const int64_t* seg, int nseg,
                 double* w, cudaStream_t s);
void scale_dev(const double* x, const double* sc, int64_t n, int nrhs, const int64_t* seg, int nseg, double* y,
               cudaStream_t s);

}  // namespace h2rs
