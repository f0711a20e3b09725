// Float64 H^2 matrix-vector product y = A x in the format of Sec. 1.1 (upsweep through
// the nested bases, couplings S_st, downsweep, dense near field) and the vector kernels
// of iterative refinement (not in the paper: it recovers float64 accuracy from a
// float32 factor).  Coefficient vectors of
// node g live at coef_off[g]*nrhs, rank_g x nrhs column-major.
#include "h2rs_internal.h"
#include "matvec.cuh"

namespace h2rs {

// Every product kernel: one thread per row of its result, RB right-hand sides per pass
// in registers (a matrix entry loaded once serves RB columns; RB = 1 for one column).
constexpr int kMvRB = 8;

template <int RB>
__global__ void mv_leaf_up(const double* __restrict__ U, const int64_t* __restrict__ U_off,
                           const int64_t* __restrict__ start, const int64_t* __restrict__ size,
                           const int64_t* __restrict__ rank, const int64_t* __restrict__ coef_off,
                           int64_t first, const double* __restrict__ x, int64_t ldx,
                           double* __restrict__ xh, int nrhs) {
    const int i = blockIdx.x;
    const int64_t g = first + i;
    const int n = (int)size[g], k = (int)rank[g];
    const double* Ui = U + U_off[i];
    const double* xi = x + start[g];
    double* out = xh + coef_off[g] * nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            double acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = 0;
            const double* u = Ui + (int64_t)a * n;
            for (int q = 0; q < n; ++q) {
                const double uv = u[q];
#pragma unroll
                for (int cc = 0; cc < RB; ++cc)
                    if (cc < cm) acc[cc] += uv * xi[q + (int64_t)(c0 + cc) * ldx];
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) out[a + (int64_t)(c0 + cc) * k] = acc[cc];
        }
    }
}

// xh_p = sum_c E_c^T xh_c for the nodes p of one level (first = first node id; the
// children of p are child0[p] and child0[p] + 1)
template <int RB>
__global__ void mv_up(const double* __restrict__ E, const int64_t* __restrict__ E_off,
                      const int64_t* __restrict__ rank, const int64_t* __restrict__ coef_off, int64_t first,
                      const int64_t* __restrict__ child0, double* __restrict__ xh, int nrhs) {
    const int64_t p = first + blockIdx.x;
    const int64_t c0n = child0[p];
    const int kp = (int)rank[p];
    double* out = xh + coef_off[p] * nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < kp; a += blockDim.x) {
            double acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = 0;
            for (int64_t ch = c0n; ch <= c0n + 1; ++ch) {
                const int kc = (int)rank[ch];
                const double* Ec = E + E_off[ch] + (int64_t)a * kc;   // column a of E_c
                const double* xc = xh + coef_off[ch] * nrhs + (int64_t)c0 * kc;
                for (int q = 0; q < kc; ++q) {
                    const double ev = Ec[q];
#pragma unroll
                    for (int cc = 0; cc < RB; ++cc)
                        if (cc < cm) acc[cc] += ev * xc[q + (int64_t)cc * kc];
                }
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) out[a + (int64_t)(c0 + cc) * kp] = acc[cc];
        }
    }
}

// yh_s = sum_{t admissible} S_st xh_t for every node s
template <int RB>
__global__ void mv_couple(const double* __restrict__ S, const int64_t* __restrict__ S_off,
                          const int64_t* __restrict__ adm_ptr, const int64_t* __restrict__ adm_col,
                          const int64_t* __restrict__ rank, const int64_t* __restrict__ coef_off,
                          const double* __restrict__ xh, double* __restrict__ yh, int nrhs) {
    const int64_t s = blockIdx.x;
    const int ks = (int)rank[s];
    double* out = yh + coef_off[s] * nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < ks; a += blockDim.x) {
            double acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = 0;
            for (int64_t q = adm_ptr[s]; q < adm_ptr[s + 1]; ++q) {
                const int64_t t = adm_col[q];
                const int kt = (int)rank[t];
                const double* St = S + S_off[q] + a;
                const double* xt = xh + coef_off[t] * nrhs + (int64_t)c0 * kt;
                for (int b = 0; b < kt; ++b) {
                    const double sv = St[(int64_t)b * ks];
#pragma unroll
                    for (int cc = 0; cc < RB; ++cc)
                        if (cc < cm) acc[cc] += sv * xt[b + (int64_t)cc * kt];
                }
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) out[a + (int64_t)(c0 + cc) * ks] = acc[cc];
        }
    }
}

// yh_c += E_c yh_parent for the nodes c of one level (roots of a forest have none)
template <int RB>
__global__ void mv_down(const double* __restrict__ E, const int64_t* __restrict__ E_off,
                        const int64_t* __restrict__ rank, const int64_t* __restrict__ coef_off, int64_t first,
                        const int64_t* __restrict__ parent, double* __restrict__ yh, int nrhs) {
    const int64_t g = first + blockIdx.x;
    const int64_t p = parent[g];
    if (p < 0) return;
    const int kc = (int)rank[g], kp = (int)rank[p];
    double* out = yh + coef_off[g] * nrhs;
    const double* yp = yh + coef_off[p] * nrhs;
    const double* Eg = E + E_off[g];
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < kc; a += blockDim.x) {
            double acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = 0;
            for (int b = 0; b < kp; ++b) {
                const double ev = Eg[a + (int64_t)b * kc];
#pragma unroll
                for (int cc = 0; cc < RB; ++cc)
                    if (cc < cm) acc[cc] += ev * yp[b + (int64_t)(c0 + cc) * kp];
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) out[a + (int64_t)(c0 + cc) * kc] += acc[cc];
        }
    }
}

// y_i = U_i yh_i + sum_{t near} D_it x_t on the leaves
template <int RB>
__global__ void mv_leaf_down(const double* __restrict__ U, const int64_t* __restrict__ U_off,
                             const double* __restrict__ D, const int64_t* __restrict__ D_off,
                             const int64_t* __restrict__ inad_ptr, const int64_t* __restrict__ inad_col,
                             const int64_t* __restrict__ start, const int64_t* __restrict__ size,
                             const int64_t* __restrict__ rank, const int64_t* __restrict__ coef_off,
                             int64_t first, const double* __restrict__ yh, const double* __restrict__ x,
                             int64_t ldx, double* __restrict__ y, int64_t ldy, int nrhs) {
    const int i = blockIdx.x;
    const int64_t g = first + i;
    const int n = (int)size[g], k = (int)rank[g];
    const double* Ui = U + U_off[i];
    const double* yi = yh + coef_off[g] * nrhs;
    const int64_t base = inad_ptr[first];
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            double acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = 0;
            for (int b = 0; b < k; ++b) {
                const double uv = Ui[a + (int64_t)b * n];
#pragma unroll
                for (int cc = 0; cc < RB; ++cc)
                    if (cc < cm) acc[cc] += uv * yi[b + (int64_t)(c0 + cc) * k];
            }
            for (int64_t q = inad_ptr[g]; q < inad_ptr[g + 1]; ++q) {
                const int64_t t = inad_col[q];
                const int nt = (int)size[t];
                const double* Dq = D + D_off[q - base] + a;
                const double* xt = x + start[t] + (int64_t)c0 * ldx;
                for (int b = 0; b < nt; ++b) {
                    const double dv = Dq[(int64_t)b * n];
#pragma unroll
                    for (int cc = 0; cc < RB; ++cc)
                        if (cc < cm) acc[cc] += dv * xt[b + (int64_t)cc * ldx];
                }
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) y[start[g] + a + (int64_t)(c0 + cc) * ldy] = acc[cc];
        }
    }
}

// r = b - y (column-major n x nrhs)
__global__ void v_residual(const double* __restrict__ b, int64_t ldb, const double* __restrict__ y,
                           int64_t ldy, double* __restrict__ r, int64_t ldr, int64_t n, int nrhs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int64_t a = e % n, c = e / n;
    r[a + c * ldr] = b[a + c * ldb] - y[a + c * ldy];
}

// x += d
__global__ void v_add(double* __restrict__ x, int64_t ldx, const double* __restrict__ d, int64_t ldd,
                      int64_t n, int nrhs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int64_t a = e % n, c = e / n;
    x[a + c * ldx] += d[a + c * ldd];
}

// Segments: the rows of system z are seg[z] .. seg[z+1]-1; channel q = c * nseg + z is
// column c restricted to system z (each channel is an independent Krylov space).
__device__ inline int seg_of(const int64_t* __restrict__ seg, int nseg, int64_t a) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg[mid] <= a) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// h[i*nq + q] = <V_i, w> over channel q (blockIdx: x = i, y = column, z = segment)
__global__ void v_multidot(const double* __restrict__ V, const double* __restrict__ w, int64_t n, int nrhs,
                           const int64_t* __restrict__ seg, int nseg, double* __restrict__ h) {
    __shared__ double red[32];
    const int i = blockIdx.x, c = blockIdx.y, z = blockIdx.z;
    const double* vi = V + ((int64_t)i * nrhs + c) * n;
    const double* wc = w + (int64_t)c * n;
    double acc = 0;
    for (int64_t a = seg[z] + threadIdx.x; a < seg[z + 1]; a += blockDim.x) acc += vi[a] * wc[a];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        h[(int64_t)i * nrhs * nseg + (int64_t)c * nseg + z] = t;
    }
}

// w += sum_{i < m} coef[i*nq + q] V_i, per channel q
__global__ void v_combine(const double* __restrict__ V, const double* __restrict__ coef, int m, int64_t n,
                          int nrhs, const int64_t* __restrict__ seg, int nseg, double* __restrict__ w) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int64_t a = e % n;
    const int c = (int)(e / n);
    const int64_t q = (int64_t)c * nseg + seg_of(seg, nseg, a);
    const int64_t nq = (int64_t)nrhs * nseg;
    double acc = w[e];
    for (int i = 0; i < m; ++i) acc += coef[i * nq + q] * V[((int64_t)i * nrhs + c) * n + a];
    w[e] = acc;
}

// y = s[q] x per channel q
__global__ void v_scale(const double* __restrict__ x, const double* __restrict__ sc, int64_t n, int nrhs,
                        const int64_t* __restrict__ seg, int nseg, double* __restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * nrhs) return;
    const int64_t a = e % n;
    y[e] = sc[(e / n) * nseg + seg_of(seg, nseg, a)] * x[e];
}

void multidot_dev(const double* V, const double* w, int m, int64_t n, int nrhs, const int64_t* seg, int nseg,
                  double* h, cudaStream_t s) {
    v_multidot<<<dim3(m, nrhs, nseg), 256, 0, s>>>(V, w, n, nrhs, seg, nseg, h);
    count_launch();
}

void combine_dev(const double* V, const double* coef, int m, int64_t n, int nrhs, const int64_t* seg, int nseg,
                 double* w, cudaStream_t s) {
    v_combine<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, s>>>(V, coef, m, n, nrhs, seg, nseg, w);
    count_launch();
}

void scale_dev(const double* x, const double* sc, int64_t n, int nrhs, const int64_t* seg, int nseg, double* y,
               cudaStream_t s) {
    v_scale<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, s>>>(x, sc, n, nrhs, seg, nseg, y);
    count_launch();
}

void residual_dev(const double* b, int64_t ldb, const double* y, int64_t ldy, double* r, int64_t ldr,
                  int64_t n, int nrhs, cudaStream_t s) {
    const unsigned g = (unsigned)((n * nrhs + 255) / 256);
    v_residual<<<g, 256, 0, s>>>(b, ldb, y, ldy, r, ldr, n, nrhs);
    count_launch();
}

void add_dev(double* x, int64_t ldx, const double* d, int64_t ldd, int64_t n, int nrhs, cudaStream_t s) {
    const unsigned g = (unsigned)((n * nrhs + 255) / 256);
    v_add<<<g, 256, 0, s>>>(x, ldx, d, ldd, n, nrhs);
    count_launch();
}

// out[c * nseg + z] = squared 2-norm of rows seg[z] .. seg[z+1]-1 of column c
__global__ void v_segnorm2(const double* __restrict__ v, int64_t ldv, const int64_t* __restrict__ seg, int nseg,
                           double* __restrict__ out) {
    __shared__ double red[32];
    const int z = blockIdx.x, c = blockIdx.y;
    double acc = 0;
    for (int64_t a = seg[z] + threadIdx.x; a < seg[z + 1]; a += blockDim.x) {
        const double t = v[a + c * ldv];
        acc += t * t;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        out[(int64_t)c * nseg + z] = s;
    }
}

void segnorm2_dev(const double* v, int64_t ldv, const int64_t* seg, int nseg, int nrhs, double* out,
                  cudaStream_t s) {
    v_segnorm2<<<dim3(nseg, nrhs), 256, 0, s>>>(v, ldv, seg, nseg, out);
    count_launch();
}

// ------------------------------------------------------------------ driver
void matvec_dev(const MatrixObj& M, int nrhs, const double* x, int64_t ldx, double* y, int64_t ldy,
                cudaStream_t s, double* scratch) {
    const HostStructure& H = M.H;
    const int d = H.d;
    const int64_t ncoef = M.coef_off.back();
    DevBuf xh_buf, yh_buf;
    double* xh_p = scratch;
    double* yh_p = scratch ? scratch + ncoef * nrhs : nullptr;
    if (!scratch) {
        xh_buf.alloc(std::max<int64_t>(1, ncoef * nrhs) * sizeof(double), s);
        yh_buf.alloc(std::max<int64_t>(1, ncoef * nrhs) * sizeof(double), s);
        xh_p = xh_buf.as<double>();
        yh_p = yh_buf.as<double>();
    }
    struct { double* p; } xh{xh_p}, yh{yh_p};
    const int64_t first_leaf = H.lev_first[d];
    const int nleaf = (int)H.lev_cnt[d];
    const int64_t* rank = M.d_rank.as<int64_t>();
    const int64_t* coef = M.d_coef_off.as<int64_t>();
    const bool one = nrhs == 1;
    if (one) mv_leaf_up<1><<<nleaf, 128, 0, s>>>(M.U.as<double>(), M.d_U_off.as<int64_t>(), M.d_node_start.as<int64_t>(),
                                                 M.d_node_size.as<int64_t>(), rank, coef, first_leaf, x, ldx, xh.p, nrhs);
    else mv_leaf_up<kMvRB><<<nleaf, 128, 0, s>>>(M.U.as<double>(), M.d_U_off.as<int64_t>(), M.d_node_start.as<int64_t>(),
                                                 M.d_node_size.as<int64_t>(), rank, coef, first_leaf, x, ldx, xh.p, nrhs);
    count_launch();
    for (int l = d; l >= 1; --l) {
        const unsigned g = (unsigned)H.lev_cnt[l - 1];
        if (one) mv_up<1><<<g, 128, 0, s>>>(M.E.as<double>(), M.d_E_off.as<int64_t>(), rank, coef, H.lev_first[l - 1],
                                            M.d_child0.as<int64_t>(), xh.p, nrhs);
        else mv_up<kMvRB><<<g, 128, 0, s>>>(M.E.as<double>(), M.d_E_off.as<int64_t>(), rank, coef, H.lev_first[l - 1],
                                            M.d_child0.as<int64_t>(), xh.p, nrhs);
        count_launch();
    }
    if (one) mv_couple<1><<<(unsigned)H.nnodes, 128, 0, s>>>(M.S.as<double>(), M.d_S_off.as<int64_t>(),
                                                             M.d_adm_ptr.as<int64_t>(), M.d_adm_col.as<int64_t>(),
                                                             rank, coef, xh.p, yh.p, nrhs);
    else mv_couple<kMvRB><<<(unsigned)H.nnodes, 128, 0, s>>>(M.S.as<double>(), M.d_S_off.as<int64_t>(),
                                                             M.d_adm_ptr.as<int64_t>(), M.d_adm_col.as<int64_t>(),
                                                             rank, coef, xh.p, yh.p, nrhs);
    count_launch();
    for (int l = 1; l <= d; ++l) {
        const unsigned g = (unsigned)H.lev_cnt[l];
        if (one) mv_down<1><<<g, 128, 0, s>>>(M.E.as<double>(), M.d_E_off.as<int64_t>(), rank, coef, H.lev_first[l],
                                              M.d_parent.as<int64_t>(), yh.p, nrhs);
        else mv_down<kMvRB><<<g, 128, 0, s>>>(M.E.as<double>(), M.d_E_off.as<int64_t>(), rank, coef, H.lev_first[l],
                                              M.d_parent.as<int64_t>(), yh.p, nrhs);
        count_launch();
    }
    if (one)
        mv_leaf_down<1><<<nleaf, 128, 0, s>>>(M.U.as<double>(), M.d_U_off.as<int64_t>(), M.D.as<double>(),
                                              M.d_D_off.as<int64_t>(), M.d_inad_ptr.as<int64_t>(),
                                              M.d_inad_col.as<int64_t>(), M.d_node_start.as<int64_t>(),
                                              M.d_node_size.as<int64_t>(), rank, coef, first_leaf, yh.p, x, ldx, y,
                                              ldy, nrhs);
    else
        mv_leaf_down<kMvRB><<<nleaf, 128, 0, s>>>(M.U.as<double>(), M.d_U_off.as<int64_t>(), M.D.as<double>(),
                                                  M.d_D_off.as<int64_t>(), M.d_inad_ptr.as<int64_t>(),
                                                  M.d_inad_col.as<int64_t>(), M.d_node_start.as<int64_t>(),
                                                  M.d_node_size.as<int64_t>(), rank, coef, first_leaf, yh.p, x, ldx,
                                                  y, ldy, nrhs);
    count_launch();
    H2_CUDA_CHECK(cudaGetLastError());
}

}  // namespace h2rs
