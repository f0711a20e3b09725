// Solve (Alg. 3): forward sweep over the levels in elimination order (Q~^T, then the
// L update per colour), diagonal L solves and upsweep; float64 dense top solve;
// downsweep, diagonal U solves and the backward sweep in reverse colour order (U
// update, then Q~).  Vectors of a level hold each box's coordinates contiguously:
// box i at offset voff[i]*nrhs, n_i x nrhs column-major.
#include "factor_impl.h"
#include "lu_solve.cuh"

namespace h2rs {

// ------------------------------------------------------------------ kernels
template <class T>
__global__ void s_load(const double* __restrict__ b, int64_t ldb, int nrhs, const int64_t* __restrict__ start,
                       const int* __restrict__ n, const int64_t* __restrict__ voff, T* __restrict__ x) {
    const int i = blockIdx.x;
    const int ni = n[i];
    T* xi = x + voff[i] * nrhs;
    const double* bi = b + start[i];
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        const int a = e % ni, c = e / ni;
        xi[e] = (T)bi[a + (int64_t)c * ldb];
    }
}

template <class T>
__global__ void s_store(double* __restrict__ b, int64_t ldb, int nrhs, const int64_t* __restrict__ start,
                        const int* __restrict__ n, const int64_t* __restrict__ voff, const T* __restrict__ x) {
    const int i = blockIdx.x;
    const int ni = n[i];
    const T* xi = x + voff[i] * nrhs;
    double* bi = b + start[i];
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) {
        const int a = e % ni, c = e / ni;
        bi[a + (int64_t)c * ldb] = (double)xi[e];
    }
}

// Right-hand sides in register blocks of RB columns: a matrix entry loaded once serves
// RB columns (RB = 1 for a single right-hand side).
constexpr int kRB = 8;

// x_i <- Q~_i^T x_i (trans = 1) or Q~_i x_i (trans = 0) for the boxes of a colour; one
// thread per row of the result, RB right-hand sides per pass.  Every solve kernel reads
// the factor in its storage type T and computes in the vector type V (T, or float64).
template <class T, class V, int RB>
__global__ void s_apply_q(const int* __restrict__ boxes, const int* __restrict__ n, const T* __restrict__ Q,
                          const int64_t* __restrict__ Q_off, const int64_t* __restrict__ voff, V* __restrict__ x,
                          int nrhs, int trans) {
    const int i = boxes[blockIdx.x];
    const int ni = n[i];
    if (ni == 0) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V* xs = reinterpret_cast<V*>(sm_raw);
    V* xi = x + voff[i] * nrhs;
    const T* Qi = Q + Q_off[i];
    for (int e = threadIdx.x; e < ni * nrhs; e += blockDim.x) xs[e] = xi[e];
    __syncthreads();
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        for (int a = threadIdx.x; a < ni; a += blockDim.x) {
            V acc[RB];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = V(0);
            for (int q = 0; q < ni; ++q) {
                const V qv = (V)(trans ? Qi[q + (int64_t)a * ni] : Qi[a + (int64_t)q * ni]);
#pragma unroll
                for (int cc = 0; cc < RB; ++cc)
                    if (cc < cm) acc[cc] += qv * xs[q + (c0 + cc) * ni];
            }
#pragma unroll
            for (int cc = 0; cc < RB; ++cc)
                if (cc < cm) xi[a + (int64_t)(c0 + cc) * ni] = acc[cc];
        }
    }
}

// forward L update of a colour, target owned: x_j -= sum_i W_L^i[j] x_{i_R}.  One block
// per target box; warp w takes every 8th column b of each contributor's W_L^i block,
// lane l accumulates rows l + 32u (RU per lane) for RB right-hand sides in registers,
// then the 8 warps are summed in shared memory (8 x m x RB of V).
template <class T, class V, int RU, int RB>
__global__ void __launch_bounds__(256)
s_fwd_l(const int* __restrict__ tbox, const int* __restrict__ tptr, const int* __restrict__ ci,
        const int* __restrict__ cpos, int cur, const int* __restrict__ colour,
        const int* __restrict__ n, const int* __restrict__ kt, const int* __restrict__ nb_ptr,
        const int* __restrict__ nbofs, const T* __restrict__ WL,
        const int64_t* __restrict__ WL_off, const int* __restrict__ WLld,
        const int64_t* __restrict__ voff, V* __restrict__ x, int nrhs) {
    const int t = blockIdx.x;
    const int j = tbox[t];
    const int nj = n[j];
    // boxes eliminated before (or in) this colour: rows j_R of W_L^i are exact zeros
    const int lo = (colour[j] <= cur) ? nj - kt[j] : 0;
    const int m = nj - lo;
    if (m <= 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V* red = reinterpret_cast<V*>(sm_raw);                 // nw x m x RB
    V* xj = x + voff[j] * nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        V acc[RU][RB];
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[u][cc] = V(0);
        for (int q = tptr[t]; q < tptr[t + 1]; ++q) {
            const int i = ci[q];
            const int ni = n[i], ri = ni - kt[i];
            if (ri <= 0) continue;
            // W_L^i holds all n_j rows of a neighbour j (skip the zero rows of an
            // eliminated j) but only the skeleton rows of i itself
            const T* W = WL + WL_off[i] + nbofs[nb_ptr[i] + cpos[q]] + (j == i ? 0 : lo);
            const int64_t ld = WLld[i];
            const V* xr = x + voff[i] * nrhs + (int64_t)c0 * ni;
            for (int b = w; b < ri; b += nw) {
                V xb[RB];
#pragma unroll
                for (int cc = 0; cc < RB; ++cc) xb[cc] = cc < cm ? xr[b + (int64_t)cc * ni] : V(0);
                const T* col = W + (int64_t)b * ld;
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int a = lane + 32 * u;
                    if (a < m) {
                        const V wv = (V)col[a];
#pragma unroll
                        for (int cc = 0; cc < RB; ++cc) acc[u][cc] += wv * xb[cc];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int a = lane + 32 * u;
            if (a < m)
#pragma unroll
                for (int cc = 0; cc < RB; ++cc) red[(w * m + a) * RB + cc] = acc[u][cc];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < m * cm; e += blockDim.x) {
            const int a = e % m, cc = e / m;
            V sacc = 0;
            for (int q = 0; q < nw; ++q) sacc += red[(q * m + a) * RB + cc];
            xj[lo + a + (int64_t)(c0 + cc) * nj] -= sacc;
        }
        __syncthreads();
    }
}

// backward U update of a colour: x_{i_R} -= sum_k W_U^i[k] x_k (box owned).  One block
// per box; warp w takes every 8th column of each neighbour segment of W_U^i, lane l
// accumulates rows l + 32u (RU per lane) for RB right-hand sides in registers, then the
// 8 warps are summed.
template <class T, class V, int RU, int RB>
__global__ void __launch_bounds__(256)
s_bwd_u(const int* __restrict__ boxes, const int* __restrict__ n, const int* __restrict__ kt,
        const int* __restrict__ nb_ptr, const int* __restrict__ nb_col,
        const int* __restrict__ nbofs, const T* __restrict__ WU,
        const int64_t* __restrict__ WU_off, const int64_t* __restrict__ voff,
        V* __restrict__ x, int nrhs) {
    const int i = boxes[blockIdx.x];
    const int ni = n[i], ri = ni - kt[i];
    if (ri <= 0) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V* red = reinterpret_cast<V*>(sm_raw);                 // 8 x ri x RB
    V* xi = x + voff[i] * nrhs;
    const T* Wi = WU + WU_off[i];
    for (int c0 = 0; c0 < nrhs; c0 += RB) {
        const int cm = min(RB, nrhs - c0);
        V acc[RU][RB];
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[u][cc] = V(0);
        for (int p = nb_ptr[i]; p < nb_ptr[i + 1]; ++p) {
            const int jb = nb_col[p];
            const int o = nbofs[p];
            const V* xs;
            int wdt, nx;
            if (jb == i) { xs = xi + (int64_t)c0 * ni + ri; wdt = kt[i]; nx = ni; }
            else { nx = n[jb]; xs = x + voff[jb] * nrhs + (int64_t)c0 * nx; wdt = nx; }
            for (int b = w; b < wdt; b += 8) {
                V xb[RB];
#pragma unroll
                for (int cc = 0; cc < RB; ++cc) xb[cc] = cc < cm ? xs[b + (int64_t)cc * nx] : V(0);
                const T* col = Wi + (int64_t)(o + b) * ri;
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int aa = lane + 32 * u;
                    if (aa < ri) {
                        const V wv = (V)col[aa];
#pragma unroll
                        for (int cc = 0; cc < RB; ++cc) acc[u][cc] += wv * xb[cc];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int aa = lane + 32 * u;
            if (aa < ri)
#pragma unroll
                for (int cc = 0; cc < RB; ++cc) red[(w * ri + aa) * RB + cc] = acc[u][cc];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ri * cm; e += blockDim.x) {
            const int aa = e % ri, cc = e / ri;
            V sacc = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) sacc += red[(q * ri + aa) * RB + cc];
            xi[aa + (int64_t)(c0 + cc) * ni] -= sacc;
        }
        __syncthreads();
    }
}

// diagonal solve with the redundant block: x_{i_R} <- D_RR^-1 x_{i_R} (the explicit
// inverse formed by the factorisation), one block per skeletonised box
template <class T, class V>
__global__ void s_diag(const int* __restrict__ boxes, const int* __restrict__ n, const int* __restrict__ kt,
                       const T* __restrict__ DI, const int64_t* __restrict__ DI_off,
                       const int64_t* __restrict__ voff, V* __restrict__ x, int nrhs) {
    const int i = boxes[blockIdx.x];
    const int ni = n[i], r = ni - kt[i];
    if (r <= 0) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    V* xs = reinterpret_cast<V*>(sm_raw);
    V* xi = x + voff[i] * nrhs;
    const T* D = DI + DI_off[i];
    for (int e = threadIdx.x; e < r * nrhs; e += blockDim.x) xs[e] = xi[(e % r) + (int64_t)(e / r) * ni];
    __syncthreads();
    for (int e = threadIdx.x; e < r * nrhs; e += blockDim.x) {
        const int a = e % r, c = e / r;
        V acc = 0;
        for (int q = 0; q < r; ++q) acc += (V)D[a + (int64_t)q * r] * xs[q + c * r];
        xi[a + (int64_t)c * ni] = acc;
    }
}

// diagonal solve by triangular solves with the LU factors (P D_RR = L U; perm in `piv`):
// x_{i_R} <- U^-1 L^-1 P x_{i_R}, one block per skeletonised box, each warp 8 right-hand
// sides in registers (lu_solve.cuh).  A warp reads all of its columns before it writes.
template <class T, class V, int RU>
__global__ void __launch_bounds__(256)
s_diag_lu(const int* __restrict__ boxes, const int* __restrict__ n, const int* __restrict__ kt,
          const T* __restrict__ LU, const int64_t* __restrict__ LU_off, const int* __restrict__ piv,
          const int64_t* __restrict__ piv_off, const int64_t* __restrict__ voff, V* __restrict__ x, int nrhs) {
    const int i = boxes[blockIdx.x];
    const int ni = n[i], r = ni - kt[i];
    if (r <= 0) return;
    const int lane = threadIdx.x & 31;
    const int* perm = piv + piv_off[i];
    const T* G = LU + LU_off[i];
    V* xi = x + voff[i] * nrhs;
    int pq[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {                         // row permutation, bounds-checked
        const int q = lane + 32 * u;
        const int pv = q < r ? perm[q] : 0;
        pq[u] = (unsigned)pv < (unsigned)r ? pv : 0;
    }
    for (int c0 = kLuCols * (threadIdx.x >> 5); c0 < nrhs; c0 += kLuCols * (blockDim.x >> 5)) {
        V v[RU][kLuCols];
#pragma unroll
        for (int c = 0; c < kLuCols; ++c)
#pragma unroll
            for (int u = 0; u < RU; ++u)
                v[u][c] = (c0 + c < nrhs && lane + 32 * u < r) ? xi[pq[u] + (int64_t)(c0 + c) * ni] : V(0);
        lu_solve_warp(v, G, r, lane);
#pragma unroll
        for (int c = 0; c < kLuCols; ++c)
#pragma unroll
            for (int u = 0; u < RU; ++u)
                if (c0 + c < nrhs && lane + 32 * u < r) xi[lane + 32 * u + (int64_t)(c0 + c) * ni] = v[u][c];
    }
}

// skeleton parts of the two children <-> parent box (up: gather, down: scatter)
template <class T>
__global__ void s_sweep(const int* __restrict__ cn, const int* __restrict__ ckt, const int64_t* __restrict__ cvoff,
                        T* __restrict__ cx, const int64_t* __restrict__ pvoff, T* __restrict__ px,
                        int nrhs, int up) {
    const int p = blockIdx.x;
    const int c1 = 2 * p, c2 = 2 * p + 1;
    const int k1 = ckt[c1], k2 = ckt[c2];
    const int np = k1 + k2;
    T* xp = px + pvoff[p] * nrhs;
    for (int e = threadIdx.x; e < np * nrhs; e += blockDim.x) {
        const int a = e % np, c = e / np;
        const int ch = a < k1 ? c1 : c2;
        const int a1 = a < k1 ? a : a - k1;
        const int nc = cn[ch];
        T* xc = cx + cvoff[ch] * nrhs + (int64_t)c * nc + (nc - ckt[ch]) + a1;
        if (up) xp[e] = *xc;
        else *xc = xp[e];
    }
}

// top boxes of one level: gather into / scatter from their system's float64 dense
// vector (system z at sys_xt[z]*nrhs, column-major nt_z x nrhs)
template <class T>
__global__ void s_top_io(const int* __restrict__ boxes, const int* __restrict__ n,
                         const int64_t* __restrict__ voff, const int64_t* __restrict__ ttoff,
                         const int* __restrict__ tsys, const TopSys* __restrict__ tops,
                         const int64_t* __restrict__ sys_xt, T* __restrict__ x, double* __restrict__ xt,
                         int nrhs, int to_dense) {
    const int p = boxes[blockIdx.x];
    const int np = n[p];
    const int z = tsys[p];
    const int64_t nt = tops[z].nt;
    T* xp = x + voff[p] * nrhs;
    double* xz = xt + sys_xt[z] * nrhs + ttoff[p];
    for (int e = threadIdx.x; e < np * nrhs; e += blockDim.x) {
        const int a = e % np, c = e / np;
        double* d = xz + a + (int64_t)c * nt;
        if (to_dense) *d = (double)xp[e];
        else xp[e] = (T)*d;
    }
}

// L_t U_t solve of every system's top matrix (blockIdx.x = column, blockIdx.y = system)
__global__ void s_top_solve(const TopSys* __restrict__ tops, const int64_t* __restrict__ sys_xt,
                            double* __restrict__ xt, int nrhs) {
    const TopSys ts = tops[blockIdx.y];
    const int64_t nt = ts.nt;
    if (nt == 0) return;
    const double* LU = ts.A;
    const int* piv = ts.piv;
    double* x = xt + sys_xt[blockIdx.y] * nrhs + (int64_t)blockIdx.x * nt;
    const int tid = threadIdx.x;
    if (tid == 0)
        for (int64_t j = 0; j < nt; ++j) {
            const int64_t p = piv[j];
            if (p < j || p >= nt) break;           // never produced by the panel kernel
            if (p != j) { const double t0 = x[j]; x[j] = x[p]; x[p] = t0; }
        }
    __syncthreads();
    for (int64_t j = 0; j < nt; ++j) {
        const double xj = x[j];
        for (int64_t a = j + 1 + tid; a < nt; a += blockDim.x) x[a] -= LU[a + j * nt] * xj;
        __syncthreads();
    }
    for (int64_t j = nt - 1; j >= 0; --j) {
        if (tid == 0) x[j] /= LU[j + j * nt];
        __syncthreads();
        const double xj = x[j];
        for (int64_t a = tid; a < j; a += blockDim.x) x[a] -= LU[a + j * nt] * xj;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ driver
template <class K>
static void allow_smem(K kern) {
    int dev = 0, optin = 0;
    H2_CUDA_CHECK(cudaGetDevice(&dev));
    H2_CUDA_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    H2_CUDA_CHECK(cudaFuncGetAttributes(&fa, kern));
    H2_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       optin - (int)fa.sharedSizeBytes));
}

template <class T, class V, int RB>
static void launch_bwd_u_rb(int nmax, int nb, cudaStream_t s, const int* boxes, const int* n, const int* kt,
                            const int* nb_ptr, const int* nb_col, const int* nbofs, const T* WU,
                            const int64_t* WU_off, const int64_t* voff, V* x, int nrhs) {
    const int smem = 8 * nmax * RB * (int)sizeof(V);
    if (nmax <= 32) s_bwd_u<T, V, 1, RB><<<nb, 256, smem, s>>>(boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
    else if (nmax <= 64) s_bwd_u<T, V, 2, RB><<<nb, 256, smem, s>>>(boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
    else if (nmax <= 128) s_bwd_u<T, V, 4, RB><<<nb, 256, smem, s>>>(boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
    else if (nmax <= 256) s_bwd_u<T, V, 8, RB><<<nb, 256, smem, s>>>(boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the solve"};
}

// backward U update: RB = 4 right-hand sides per pass (RU rows per lane x RB registers)
template <class T, class V>
static void launch_bwd_u(int nmax, int nb, cudaStream_t s, const int* boxes, const int* n, const int* kt,
                         const int* nb_ptr, const int* nb_col, const int* nbofs, const T* WU,
                         const int64_t* WU_off, const int64_t* voff, V* x, int nrhs) {
    if (nrhs == 1) launch_bwd_u_rb<T, V, 1>(nmax, nb, s, boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
    else launch_bwd_u_rb<T, V, 4>(nmax, nb, s, boxes, n, kt, nb_ptr, nb_col, nbofs, WU, WU_off, voff, x, nrhs);
}

template <class T, class V>
static void launch_diag_lu(int nmax, unsigned nb, cudaStream_t s, const int* boxes, const int* n, const int* kt,
                           const T* LU, const int64_t* LU_off, const int* piv, const int64_t* piv_off,
                           const int64_t* voff, V* x, int nrhs) {
    const int th = 32 * std::min(8, (nrhs + kLuCols - 1) / kLuCols);
    if (nmax <= 32) s_diag_lu<T, V, 1><<<nb, th, 0, s>>>(boxes, n, kt, LU, LU_off, piv, piv_off, voff, x, nrhs);
    else if (nmax <= 64) s_diag_lu<T, V, 2><<<nb, th, 0, s>>>(boxes, n, kt, LU, LU_off, piv, piv_off, voff, x, nrhs);
    else if (nmax <= 128) s_diag_lu<T, V, 4><<<nb, th, 0, s>>>(boxes, n, kt, LU, LU_off, piv, piv_off, voff, x, nrhs);
    else if (nmax <= 256) s_diag_lu<T, V, 8><<<nb, th, 0, s>>>(boxes, n, kt, LU, LU_off, piv, piv_off, voff, x, nrhs);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the solve"};
}

template <class T, class V>
static void launch_apply_q(int nb, int smem, cudaStream_t s, const int* boxes, const int* n, const T* Q,
                           const int64_t* Q_off, const int64_t* voff, V* x, int nrhs, int trans) {
    if (nrhs == 1) s_apply_q<T, V, 1><<<nb, 256, smem, s>>>(boxes, n, Q, Q_off, voff, x, nrhs, trans);
    else s_apply_q<T, V, kRB><<<nb, 256, smem, s>>>(boxes, n, Q, Q_off, voff, x, nrhs, trans);
}

template <class T, class V, int RB>
static void launch_fwd_l_rb(int nmax, int nt, cudaStream_t s, const int* tbox, const int* tptr, const int* ci,
                            const int* cpos, int cur, const int* colour, const int* n, const int* kt,
                            const int* nb_ptr, const int* nbofs, const T* WL, const int64_t* WL_off,
                            const int* WLld, const int64_t* voff, V* x, int nrhs) {
    const int smem = 8 * nmax * RB * (int)sizeof(V);
#define H2_FWD_L(RU) s_fwd_l<T, V, RU, RB><<<nt, 256, smem, s>>>(tbox, tptr, ci, cpos, cur, colour, n, kt, nb_ptr, \
                                                                 nbofs, WL, WL_off, WLld, voff, x, nrhs)
    if (nmax <= 32) H2_FWD_L(1);
    else if (nmax <= 64) H2_FWD_L(2);
    else if (nmax <= 128) H2_FWD_L(4);
    else if (nmax <= 256) H2_FWD_L(8);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the solve"};
#undef H2_FWD_L
}

// forward L update: RB = 4 right-hand sides per pass, nmax bounds the target sizes
template <class T, class V>
static void launch_fwd_l(int nmax, int nt, cudaStream_t s, const int* tbox, const int* tptr, const int* ci,
                         const int* cpos, int cur, const int* colour, const int* n, const int* kt,
                         const int* nb_ptr, const int* nbofs, const T* WL, const int64_t* WL_off, const int* WLld,
                         const int64_t* voff, V* x, int nrhs) {
    if (nrhs == 1)
        launch_fwd_l_rb<T, V, 1>(nmax, nt, s, tbox, tptr, ci, cpos, cur, colour, n, kt, nb_ptr, nbofs, WL, WL_off,
                                 WLld, voff, x, nrhs);
    else
        launch_fwd_l_rb<T, V, 4>(nmax, nt, s, tbox, tptr, ci, cpos, cur, colour, n, kt, nb_ptr, nbofs, WL, WL_off,
                                 WLld, voff, x, nrhs);
}

template <class T, class V>
static void allow_solve_smem() {
    static bool ready = false;
    if (ready) return;
    allow_smem(s_apply_q<T, V, 1>);
    allow_smem(s_apply_q<T, V, kRB>);
    allow_smem(s_diag<T, V>);
    allow_smem(s_bwd_u<T, V, 8, 1>);
    allow_smem(s_bwd_u<T, V, 8, 4>);
    allow_smem(s_bwd_u<T, V, 4, 4>);
    allow_smem(s_bwd_u<T, V, 2, 4>);
    allow_smem(s_bwd_u<T, V, 1, 4>);
    allow_smem(s_fwd_l<T, V, 8, 4>);
    allow_smem(s_fwd_l<T, V, 4, 4>);
    allow_smem(s_fwd_l<T, V, 2, 4>);
    allow_smem(s_fwd_l<T, V, 1, 4>);
    allow_smem(s_fwd_l<T, V, 8, 1>);
    ready = true;
}

template <class T>
void FactorImpl<T>::solve_dev(double* b, int nrhs, int64_t ldb, bool wide) {
    if (wide) solve_in<double>(b, nrhs, ldb);
    else solve_in<T>(b, nrhs, ldb);
}

// The solve with vectors and arithmetic in V over the factor stored in T.
template <class T>
template <class V>
void FactorImpl<T>::solve_in(double* b, int nrhs, int64_t ldb) {
    cudaStream_t s = stream;
    allow_solve_smem<T, V>();
    const Plan& P = A->plan;
    const size_t nl = P.levels.size();
    std::vector<DevBuf> vec(nl + 1);
    for (size_t a = 0; a <= nl; ++a)
        vec[a].alloc(std::max<int64_t>(1, lv[a].vtot * nrhs) * sizeof(V), s);
    // leaf starts (tree order) of the first level's boxes
    LevelRT& L0 = lv[0];
    DevBuf d_start;
    {
        std::vector<int64_t> st(L0.cnt);
        for (int i = 0; i < L0.cnt; ++i) st[i] = A->H.node_start[L0.S->first + i];
        upload(d_start, st, s);
    }
    s_load<V><<<L0.cnt, 256, 0, s>>>(b, ldb, nrhs, d_start.as<int64_t>(), L0.d_n.as<int>(),
                                     L0.d_voff.as<int64_t>(), vec[0].as<V>());
    count_launch();
    // boxes of each colour: the plan's device list, colour c at cbox_ptr[c]
    // forward
    for (size_t a = 0; a < nl; ++a) {
        LevelRT& L = lv[a];
        const LevelStruct& S = *L.S;
        int nmax = 1, nall = 1;
        for (int i : S.skel_boxes) nmax = std::max(nmax, L.n[i]);
        for (int v : L.n) nall = std::max(nall, v);               // bound of the L-update targets
        const int qsm = nmax * nrhs * (int)sizeof(V);
        for (int c = 0; c < S.ncolour; ++c) {
            const int b0 = S.cbox_ptr[c], nb = S.cbox_ptr[c + 1] - b0;
            launch_apply_q<T, V>(nb, qsm, s, S.dev.cboxes.as<int>() + b0, L.d_n.as<int>(), L.Q.as<T>(),
                                 L.d_Q_off.as<int64_t>(), L.d_voff.as<int64_t>(), vec[a].as<V>(), nrhs, 1);
            count_launch();
            const int t0 = S.fl_cptr[c], nt_ = S.fl_cptr[c + 1] - t0;
            if (nt_) {
                launch_fwd_l<T, V>(nall, nt_, s, L.d_fl_tbox.as<int>() + t0, L.d_fl_tptr.as<int>() + t0,
                                   L.d_fl_ci.as<int>(), L.d_fl_cpos.as<int>(), c, L.d_colour.as<int>(),
                                   L.d_n.as<int>(), L.d_kt.as<int>(), L.d_nb_ptr.as<int>(), L.d_nbofs.as<int>(),
                                   L.WL.as<T>(), L.d_WL_off.as<int64_t>(), L.d_WLld.as<int>(),
                                   L.d_voff.as<int64_t>(), vec[a].as<V>(), nrhs);
                count_launch();
            }
        }
        if (!S.skel_boxes.empty()) {
            const unsigned nsk = (unsigned)S.skel_boxes.size();
            if (w_inverse)                         // explicit inverse (GEMV)
                s_diag<T, V><<<nsk, 256, nmax * nrhs * (int)sizeof(V), s>>>(
                    L.d_skel_boxes.as<int>(), L.d_n.as<int>(), L.d_kt.as<int>(), L.DI.as<T>(),
                    L.d_Q_off.as<int64_t>(), L.d_voff.as<int64_t>(), vec[a].as<V>(), nrhs);
            else
                launch_diag_lu<T, V>(nmax, nsk, s, L.d_skel_boxes.as<int>(), L.d_n.as<int>(), L.d_kt.as<int>(),
                                     L.LU.as<T>(), L.d_LU_off.as<int64_t>(), L.piv.as<int>(),
                                     L.d_piv_off.as<int64_t>(), L.d_voff.as<int64_t>(), vec[a].as<V>(), nrhs);
            count_launch();
        }
        LevelRT& Pn = lv[a + 1];
        s_sweep<V><<<Pn.cnt, 256, 0, s>>>(L.d_n.as<int>(), L.d_kt.as<int>(), L.d_voff.as<int64_t>(),
                                          vec[a].as<V>(), Pn.d_voff.as<int64_t>(), vec[a + 1].as<V>(),
                                          nrhs, 1);
        count_launch();
    }
    // dense top solves of every system (their boxes sit at the levels where each
    // system's skeletonisation ended)
    if (nt > 0) {
        DevBuf xt;
        xt.alloc(nt * nrhs * sizeof(double), s);
        for (int dir = 1; dir >= 0; --dir) {
            if (dir == 0) {
                s_top_solve<<<dim3(nrhs, (unsigned)tops.size()), 1024, 0, s>>>(
                    d_tops.as<TopSys>(), d_sys_xt.as<int64_t>(), xt.as<double>(), nrhs);
                count_launch();
            }
            for (size_t a = 0; a <= nl; ++a) {
                LevelRT& L = lv[a];
                const int ntb = (int)L.S->top_boxes.size();
                if (!ntb) continue;
                s_top_io<V><<<ntb, 256, 0, s>>>(L.d_top_boxes.as<int>(), L.d_n.as<int>(), L.d_voff.as<int64_t>(),
                                                L.d_ttoff.as<int64_t>(), L.d_tsys.as<int>(), d_tops.as<TopSys>(),
                                                d_sys_xt.as<int64_t>(), vec[a].as<V>(), xt.as<double>(), nrhs,
                                                dir);
                count_launch();
            }
        }
    }
    // backward
    for (size_t a = nl; a-- > 0;) {
        LevelRT& L = lv[a];
        const LevelStruct& S = *L.S;
        LevelRT& Pn = lv[a + 1];
        s_sweep<V><<<Pn.cnt, 256, 0, s>>>(L.d_n.as<int>(), L.d_kt.as<int>(), L.d_voff.as<int64_t>(),
                                          vec[a].as<V>(), Pn.d_voff.as<int64_t>(), vec[a + 1].as<V>(),
                                          nrhs, 0);
        count_launch();

        int nmax = 1;
        for (int i : S.skel_boxes) nmax = std::max(nmax, L.n[i]);
        const int qsm = nmax * nrhs * (int)sizeof(V);
        for (int c = S.ncolour - 1; c >= 0; --c) {
            const int b0 = S.cbox_ptr[c], nb = S.cbox_ptr[c + 1] - b0;
            launch_bwd_u<T, V>(nmax, nb, s, S.dev.cboxes.as<int>() + b0, L.d_n.as<int>(), L.d_kt.as<int>(),
                               L.d_nb_ptr.as<int>(), L.d_nb_col.as<int>(), L.d_nbofs.as<int>(),
                               L.WU.as<T>(), L.d_WU_off.as<int64_t>(), L.d_voff.as<int64_t>(),
                               vec[a].as<V>(), nrhs);
            count_launch();
            launch_apply_q<T, V>(nb, qsm, s, S.dev.cboxes.as<int>() + b0, L.d_n.as<int>(), L.Q.as<T>(),
                                 L.d_Q_off.as<int64_t>(), L.d_voff.as<int64_t>(), vec[a].as<V>(), nrhs, 0);
            count_launch();
        }
    }
    s_store<V><<<L0.cnt, 256, 0, s>>>(b, ldb, nrhs, d_start.as<int64_t>(), L0.d_n.as<int>(),
                                      L0.d_voff.as<int64_t>(), vec[0].as<V>());
    count_launch();
    H2_CUDA_CHECK(cudaGetLastError());
}

template void FactorImpl<double>::solve_dev(double*, int, int64_t, bool);
template void FactorImpl<float>::solve_dev(double*, int, int64_t, bool);

}  // namespace h2rs
