// Factorisation kernels (Alg. 2 per colour, level close, top-level LU).
// Included by factor.cu only: a kernel is compiled in the translation unit that
// launches it.
//
// All per-box kernels run one thread block per box of the colour; box data
// (blocks, bases, factors) sit at prefix-sum offsets inside per-level buffers
// (Sec. 2.2: no per-box allocation).  Shapes are data dependent (augmented ranks are
// only known on the device), so every kernel reads n_i and k~_i from device arrays.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "factor_args.cuh"
#include "lu_solve.cuh"
#include "proj_tc.cuh"
#include "schur_ws.cuh"

namespace h2rs {

// ------------------------------------------------------------------ helpers
__device__ inline void dev_fail(DevStatus* st, int code, int level, int box) {
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->level = level;
        st->box = box;
    }
}

template <class T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum; every thread gets the result.  red: 33 T of shared memory.
template <class T>
__device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T x = lane < nw ? red[lane] : T(0);
        x = warp_sum(x);
        if (lane == 0) red[32] = x;
    }
    __syncthreads();
    return red[32];
}

template <class T> __device__ inline T t_abs(T x) { return x < T(0) ? -x : x; }
template <class T> __device__ inline bool t_finite(T x) { return isfinite((double)x); }

// ================================================================== leaf load
// The dense part D of A = H + D on the leaf level (Sec. 2.1), float64 -> working
// precision, into the level's block buffer.
template <class T>
__global__ void k_leaf_load(LevelArgs<T> a, const double* __restrict__ D,
                            const int64_t* __restrict__ D_off,
                            const int64_t* __restrict__ near_entry) {
    const int b = blockIdx.x;
    const int i = a.brow[b], j = a.bcol[b];
    const int64_t cnt = (int64_t)a.n[i] * a.n[j];
    T* dst = a.blk + a.blk_off[b];
    const int64_t e = near_entry[b];
    if (e < 0) {
        for (int64_t x = threadIdx.x; x < cnt; x += blockDim.x) dst[x] = T(0);
        return;
    }
    const double* src = D + D_off[e];
    for (int64_t x = threadIdx.x; x < cnt; x += blockDim.x) dst[x] = (T)src[x];
}

// Leaf bases V_i = U_i of the given H^2 matrix (Sec. 1.1) in the working precision.
template <class T>
__global__ void k_leaf_basis(LevelArgs<T> a, T* V, const double* __restrict__ U,
                             const int64_t* __restrict__ U_off) {
    const int i = blockIdx.x;
    const int64_t cnt = (int64_t)a.n[i] * a.k[i];
    const double* src = U + U_off[i];
    T* dst = V + a.V_off[i];
    for (int64_t x = threadIdx.x; x < cnt; x += blockDim.x) dst[x] = (T)src[x];
}

// ================================================================== augmentation
// Whether box i's fill rows can be skipped: sigma_max(Y) <= ||Y||_F, so when the
// Frobenius norm is below eps_fill the truncated SVD keeps nothing (the margin covers
// the rounding of the norm itself); with forced ranks (debug) when none is asked for.
template <class T>
__device__ inline bool fill_below(const LevelArgs<T>& a, int i, double ynorm2, T eps_fill) {
    if (a.force_kt) return a.force_kt[i] - a.k[i] <= 0;
    return ynorm2 <= (double)eps_fill * (double)eps_fill * (1.0 - 4e-6);
}

// Y = (I - V V^T) F for the live columns of one fill block of box i; Y^T is written
// into the box's scratch rows (Alg. 2 truncSVD input).
// The live rows of all the box's segments are stored back to back (segment order), so
// that the R-factor streams full chunks across segment boundaries.  L.seg_j is offset to
// this colour's first segment s0; L.seg_ptr holds global segment indices.
// PC columns of F at a time; V is staged in shared memory when VS (ld n + 1), the
// chunk of F (ld n + 1) and P = V^T F (ld k + 1) always are (padded: no bank conflicts).
template <class T, bool VS>
__global__ void k_aug_gather(LevelArgs<T> a, ColourLists L, int cur, const int* __restrict__ seg_slot,
                             int s0, int PC, T* __restrict__ scratch) {
    const int s = blockIdx.x;
    const int slot = seg_slot[s];
    const int i = L.boxes[slot];
    const int b = L.seg_blk[s], j = L.seg_j[s];
    const int n = a.n[i], k = a.k[i], nj = a.n[j];
    const int skip = (a.colour[j] < cur) ? (nj - a.kt[j]) : 0;
    int64_t lp = 0;                                  // live rows of the box's earlier segments
    for (int g = L.seg_ptr[slot]; g < s0 + s; ++g) {
        const int jg = L.seg_j[g - s0];
        lp += (a.colour[jg] < cur) ? a.kt[jg] : a.n[jg];
    }
    const T* F = a.blk + a.blk_off[b];
    const T* Vg = a.V + a.V_off[i];
    const int64_t ld = L.ylead[slot];
    T* Yt = scratch + L.ybase[slot] + lp - skip;      // row c of the segment at lp + c - skip
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int lf = n + 1, lq = k + 1;
    T* Fs = reinterpret_cast<T*>(sm_raw);             // PC x (n+1): column c at c * lf
    T* Ps = Fs + (size_t)lf * PC;                     // PC x (k+1)
    T* Vs = Ps + (size_t)lq * PC;                     // k x (n+1) when VS
    const int tid = threadIdx.x, bs = blockDim.x;
    if (VS) {
        for (int x = tid; x < n * k; x += bs) Vs[(x % n) + (x / n) * lf] = Vg[x];
    }
    const T* V = VS ? Vs : Vg;
    const int lv = VS ? lf : n;
    double y2 = 0;                                   // this thread's part of ||Y||_F^2
    for (int c0 = skip; c0 < nj; c0 += PC) {
        const int pc = min(PC, nj - c0);
        for (int x = tid; x < n * pc; x += bs) {
            const int r = x % n, c = x / n;
            Fs[r + c * lf] = F[r + (int64_t)(c0 + c) * n];
        }
        __syncthreads();
        for (int x = tid; x < k * pc; x += bs) {         // P = V^T F
            const int r = x % k, c = x / k;
            const T* vr = V + (int64_t)r * lv;
            const T* fc = Fs + c * lf;
            T acc = 0;
            for (int q = 0; q < n; ++q) acc += vr[q] * fc[q];
            Ps[r + c * lq] = acc;
        }
        __syncthreads();
        for (int x = tid; x < n * pc; x += bs) {         // Y^T rows: F - V P (coalesced on c)
            const int c = x % pc, r = x / pc;
            T acc = Fs[r + c * lf];
            const T* pcol = Ps + c * lq;
            for (int q = 0; q < k; ++q) acc -= V[r + (int64_t)q * lv] * pcol[q];
            Yt[(c0 + c) + (int64_t)r * ld] = acc;
            y2 += (double)acc * (double)acc;
        }
        __syncthreads();
    }
    __shared__ double red[33];
    const double tot = block_sum(y2, red);
    if (tid == 0) atomicAdd(&L.ynorm2[slot], tot);
}

// R-factor of the live rows of Y^T (stored back to back, `live` rows) accumulated in W
// (row-major n x n, row stride ldw), streamed in chunks of 64 rows (Householder QR of
// [R; chunk] per chunk).  256 threads: 32 column groups of CPT consecutive columns x 8
// row groups; thread (g, h) keeps rows h + 8q (q < 8) of its CPT columns in registers,
// so one broadcast reflector value serves CPT columns, and the 8 row groups of a
// column group are 8 consecutive lanes (partial dot products reduced by shuffles).
// Per column the owning lanes publish the reflector and its scalars (computed once)
// through shared memory (double buffered, one barrier per column).  Requires
// n <= 32 * CPT and blockDim.x == 256.
// elements of the chunk buffer of k_basis (also holds rfactor_stream's broadcasts)
__host__ __device__ inline int basis_chunk_elems(int n) {
    const int ch = n <= 192 ? 64 : 32;
    const int e = (ch + 1) * n;
    return e > 288 ? e : 288;
}

template <class T, int CPT>
__device__ void rfactor_stream(int n, int64_t live, const T* __restrict__ Yt, int64_t ld, T* W, int ldw, T* vb) {
    constexpr int CH = 64, RG = 8, RPT = CH / RG;
    const int tid = threadIdx.x;
    const int h = tid & (RG - 1);                    // row group: rows h + RG q
    const int g = tid >> 3;                          // column group: columns CPT g + cc
    // vb: 2 buffers of [CH reflector values | tw | inv]
    constexpr int bufsz = CH + 2;
    T x[RPT][CPT];
    for (int64_t r0 = 0; r0 < live; r0 += CH) {
        const int rows = (int)min((int64_t)CH, live - r0);
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                const int rr = h + RG * q, col = CPT * g + cc;
                x[q][cc] = (rr < rows && col < n) ? Yt[(r0 + rr) + (int64_t)col * ld] : T(0);
            }
        for (int jj = 0; jj < n; ++jj) {
            T* buf = vb + (jj & 1) * bufsz;
            if (g == jj / CPT) {                         // the 8 lanes owning column jj
                const int c0 = jj % CPT;
                T p2 = 0;
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    T v = x[q][0];
#pragma unroll
                    for (int cc = 1; cc < CPT; ++cc)
                        if (cc == c0) v = x[q][cc];
                    buf[h + RG * q] = v;
                    p2 += v * v;
                }
                // only these 8 lanes of the warp take part: the mask names exactly them
                const unsigned grp = 0xffu << (8 * ((threadIdx.x & 31) >> 3));
#pragma unroll
                for (int o = 1; o < RG; o <<= 1) p2 += __shfl_xor_sync(grp, p2, o);
                if (h == 0) {
                    T tw = 0, inv = 0;
                    if (p2 != T(0)) {
                        const T x0 = W[(int64_t)jj * ldw + jj];
                        const T nrm = sqrt(x0 * x0 + p2);
                        const T beta = x0 > T(0) ? -nrm : nrm;
                        const T v0 = x0 - beta;
                        tw = -v0 / beta;
                        inv = T(1) / v0;
                        W[(int64_t)jj * ldw + jj] = beta;
                    }
                    buf[CH] = tw;
                    buf[CH + 1] = inv;
                }
            }
            __syncthreads();
            const T tw = buf[CH];
            if (tw == T(0)) continue;                    // uniform; buffers alternate
            const T inv = buf[CH + 1];
            T vr[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) vr[q] = buf[h + RG * q];
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                const int col = CPT * g + cc;
                T d = 0;
#pragma unroll
                for (int q = 0; q < RPT; ++q) d += vr[q] * x[q][cc];
#pragma unroll
                for (int o = 1; o < RG; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                if (col > jj && col < n) {
                    const T w = W[(int64_t)jj * ldw + col] + d * inv;
                    const T tww = tw * w;
                    const T f = tww * inv;
#pragma unroll
                    for (int q = 0; q < RPT; ++q) x[q][cc] -= f * vr[q];
                    if (h == 0) W[(int64_t)jj * ldw + col] -= tww;
                }
            }
        }
        __syncthreads();
    }
}

// Alg. 2, first loop, per box: R-factor of Y^T (Householder, streamed), SVD of R by
// one-sided Jacobi and truncation at eps_fill (Sec. 2.1, the second of its three ways),
// V~ = [V, Vbar] and its completion Q~ = [V~perp, V~].
// BIG: boxes up to 256 (one CTA per SM: 64 rows per thread in the R-factor); otherwise
// boxes up to 128, register-capped so that two boxes share an SM.
template <class T, bool BIG>
__global__ void __launch_bounds__(256, BIG ? 1 : 2)
k_basis(LevelArgs<T> a, ColourLists L, int cur, const T* __restrict__ scratch,
        T* __restrict__ gwork, int w_in_smem) {
    const int slot = blockIdx.x;
    const int i = L.boxes[slot];
    const int n = a.n[i], k = a.k[i];
    const T eps_fill = a.eps_fill[i];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarp = blockDim.x >> 5;
    const int CH = (n <= 192) ? 64 : 32;
    const int ldc = CH + 1;                         // padded: no bank conflicts across columns
    const int ldw = n + 1;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* C = reinterpret_cast<T*>(sm_raw);            // CH x n chunk (col-major, ld ldc)
    T* tau = C + basis_chunk_elems(n);              // n
    T* sig = tau + n;                               // n
    T* red = sig + n;                               // 33
    int* ired = reinterpret_cast<int*>(red + 33);   // 4
    T* W = w_in_smem ? reinterpret_cast<T*>(ired + 4) : gwork + L.wbase[slot];
    T* Qs = a.Q + a.Q_off[i];
    const T* V = a.V + a.V_off[i];
    const int64_t ld = L.ylead[slot];
    const T* Yt = scratch + L.ybase[slot];

    // live fill rows of this box
    const int s0 = L.seg_ptr[slot], s1 = L.seg_ptr[slot + 1];
    int64_t live = 0;
    for (int s = s0; s < s1; ++s) {
        const int j = L.seg_j[s];
        const int nj = a.n[j];
        live += nj - ((a.colour[j] < cur) ? (nj - a.kt[j]) : 0);
    }
    int keep = 0;
    // sigma_max(Y) <= ||Y||_F: when the Frobenius norm (accumulated in float64 by the
    // gather, which then stores no Y) is below eps_fill, no singular value exceeds it
    // and the truncated SVD keeps nothing, so the R-factor and the SVD are skipped
    // forced ranks (debug): keep exactly force_kt - k vectors, whatever their size
    const int fkeep = a.force_kt ? max(0, min(a.force_kt[i] - k, n - k)) : -1;
    const bool below = fill_below(a, i, L.ynorm2[slot], eps_fill);   // the gather's decision
    if (live > 0 && k < n && !below) {
        // ---------------- R-factor of Y^T (R row-major in W, row stride ldw)
        for (int x = tid; x < n * ldw; x += blockDim.x) W[x] = T(0);
        __syncthreads();
        if (n <= 32) rfactor_stream<T, 1>(n, live, Yt, ld, W, ldw, C);
        else if (n <= 64) rfactor_stream<T, 2>(n, live, Yt, ld, W, ldw, C);
        else if (!BIG || n <= 128) rfactor_stream<T, 4>(n, live, Yt, ld, W, ldw, C);
        else rfactor_stream<T, BIG ? 8 : 4>(n, live, Yt, ld, W, ldw, C);   // n <= 256
        __syncthreads();
        // ---------------- one-sided Jacobi on M = R^T (column p of M = row p of R)
        // Round-robin pairs over the active columns, tpp threads per pair (rows
        // interleaved).  Each sweep first drops columns whose squared norm is below
        // defl^2: even all of them together stay under 1e-3 eps_fill (1e-6 in float64),
        // so they cannot change which singular values exceed eps_fill; the remaining
        // columns are ordered by decreasing norm (faster convergence).
        const int meff = (int)(live < (int64_t)n ? live : (int64_t)n);
        int* act = reinterpret_cast<int*>(tau);          // active columns
        int* nact = reinterpret_cast<int*>(C);           // next sweep's active columns
        const T tol = T(n) * Eps<T>::v;
        const T defl = (sizeof(T) == 4 ? T(1e-3) : T(1e-6)) * eps_fill / sqrt(T(n));
        const T defl2 = defl * defl;
        if (tid == 0) ired[2] = meff;
        for (int p = tid; p < meff; p += blockDim.x) act[p] = p;
        __syncthreads();
        for (int sweep = 0; sweep < 40; ++sweep) {
            const int mcur = ired[2];
            for (int q = wid; q < mcur; q += nwarp) {
                const int p = act[q];
                T s2 = 0;
                for (int r = lane; r < n; r += 32) s2 += W[(int64_t)p * ldw + r] * W[(int64_t)p * ldw + r];
                s2 = warp_sum(s2);
                if (lane == 0) sig[p] = s2;
            }
            __syncthreads();
            for (int q = tid; q < mcur; q += blockDim.x) {
                const int p = act[q];
                const T sp = sig[p];
                if (sp >= defl2) {
                    int rank = 0;
                    for (int q2 = 0; q2 < mcur; ++q2) {
                        const int p2 = act[q2];
                        const T s2 = sig[p2];
                        rank += (s2 >= defl2) && (s2 > sp || (s2 == sp && p2 < p));
                    }
                    nact[rank] = p;
                }
            }
            if (tid == 0) {
                int c = 0;
                for (int q = 0; q < mcur; ++q) c += sig[act[q]] >= defl2;
                ired[3] = c;
                ired[0] = 0;
            }
            __syncthreads();
            const int ma = ired[3];
            for (int q = tid; q < ma; q += blockDim.x) act[q] = nact[q];
            if (tid == 0) ired[2] = ma;
            __syncthreads();
            const int m = ma + (ma & 1);
            const int npair = m / 2;
            if (npair == 0) break;
            int tpp = 1;
            while (tpp * 2 <= 32 && tpp * 2 * npair <= 256) tpp *= 2;
            const int pstep = 256 / tpp, ppart = tid % tpp, pofs = tid / tpp;
            int rot = 0;
            for (int round = 0; round < m - 1; ++round) {
                for (int pb = 0; pb < npair; pb += pstep) {          // uniform trip count
                    const int pr = pb + pofs;
                    const int x1 = pr, x2 = m - 1 - pr;
                    const int px = x1 == 0 ? 0 : ((x1 - 1 + round) % (m - 1)) + 1;
                    const int qx = x2 == 0 ? 0 : ((x2 - 1 + round) % (m - 1)) + 1;
                    const bool on = pr < npair && px < ma && qx < ma;
                    T* Mp = W + (int64_t)(on ? act[px] : 0) * ldw;
                    T* Mq = W + (int64_t)(on ? act[qx] : 0) * ldw;
                    T al = 0, be = 0, ga = 0;
                    if (on)
                        for (int r = ppart; r < n; r += tpp) {
                            const T u = Mp[r], v = Mq[r];
                            al += u * u; be += v * v; ga += u * v;
                        }
                    for (int o = 1; o < tpp; o <<= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    if (on && al > T(0) && be > T(0) && t_abs(ga) > tol * sqrt(al * be)) {
                        const T zeta = (be - al) / (T(2) * ga);
                        const T t = (zeta >= T(0) ? T(1) : T(-1)) /
                                    (t_abs(zeta) + sqrt(T(1) + zeta * zeta));
                        const T c = T(1) / sqrt(T(1) + t * t);
                        const T sn = c * t;
                        for (int r = ppart; r < n; r += tpp) {
                            const T u = Mp[r], v = Mq[r];
                            Mp[r] = c * u - sn * v;
                            Mq[r] = sn * u + c * v;
                        }
                        rot = 1;
                    }
                }
                __syncthreads();
            }
            if (rot) atomicOr(&ired[0], 1);
            __syncthreads();
            if (ired[0] == 0) break;
            __syncthreads();
        }
        // ---------------- singular values, selection (largest first)
        for (int p = wid; p < meff; p += nwarp) {
            T s2 = 0;
            for (int r = lane; r < n; r += 32) s2 += W[(int64_t)p * ldw + r] * W[(int64_t)p * ldw + r];
            s2 = warp_sum(s2);
            if (lane == 0) sig[p] = sqrt(s2);
        }
        __syncthreads();
        if (tid == 0) {
            int cnt = 0;
            for (int p = 0; p < meff; ++p) cnt += sig[p] > eps_fill;
            ired[1] = fkeep >= 0 ? min(fkeep, meff) : min(cnt, n - k);
        }
        __syncthreads();
        keep = ired[1];
        // stage Vbar (unnormalised order by rank) in the last keep columns of Q~
        for (int p = wid; p < meff; p += nwarp) {
            const T sp = sig[p];
            int rank = 0;
            for (int q = 0; q < meff; ++q) rank += (sig[q] > sp) || (sig[q] == sp && q < p);
            if (rank < keep) {
                T* dst = Qs + (int64_t)(n - keep + rank) * n;
                const T inv = T(1) / sp;
                for (int r = lane; r < n; r += 32) dst[r] = W[(int64_t)p * ldw + r] * inv;
            }
        }
        __syncthreads();
    }
    // ---------------- Householder QR of V~ = [V, Vbar] (n x kt) in W
    const int kt = k + keep;
    const int r_red = n - kt;
    for (int x = tid; x < n * kt; x += blockDim.x) {
        const int row = x % n, col = x / n;
        W[x] = col < k ? V[row + (int64_t)col * n] : Qs[row + (int64_t)(n - keep + col - k) * n];
    }
    __syncthreads();
    for (int jj = 0; jj < kt; ++jj) {
        T part = 0;
        for (int r = jj + 1 + tid; r < n; r += blockDim.x) part += W[r + (int64_t)jj * n] * W[r + (int64_t)jj * n];
        const T ss = block_sum(part, red);
        const T x0 = W[jj + (int64_t)jj * n];
        if (ss == T(0)) {
            if (tid == 0) tau[jj] = T(0);
            __syncthreads();
            continue;
        }
        const T nrm = sqrt(x0 * x0 + ss);
        const T beta = x0 > T(0) ? -nrm : nrm;
        const T v0 = x0 - beta;
        const T tw = -v0 / beta;
        for (int r = jj + 1 + tid; r < n; r += blockDim.x) W[r + (int64_t)jj * n] /= v0;
        __syncthreads();
        for (int col = jj + 1 + wid; col < kt; col += nwarp) {
            T w = 0;
            for (int r = jj + 1 + lane; r < n; r += 32) w += W[r + (int64_t)jj * n] * W[r + (int64_t)col * n];
            w = warp_sum(w) + W[jj + (int64_t)col * n];
            const T tww = tw * w;
            for (int r = jj + 1 + lane; r < n; r += 32) W[r + (int64_t)col * n] -= tww * W[r + (int64_t)jj * n];
            if (lane == 0) W[jj + (int64_t)col * n] -= tww;
        }
        __syncthreads();
        if (tid == 0) {
            tau[jj] = tw;
            W[jj + (int64_t)jj * n] = beta;
        }
        __syncthreads();
    }
    // Q_h[:, k + t], t in [0, n-k): t < keep -> Vbar (Q~ col r+k+t), else V~perp (col t-keep)
    const int nout = n - k;
    const int cw = CH;                               // columns per chunk (C holds n x CH)
    for (int t0 = 0; t0 < nout; t0 += cw) {
        const int tw_ = min(cw, nout - t0);
        for (int x = tid; x < n * tw_; x += blockDim.x) {
            const int row = x % n, t = x / n;
            C[row + (int64_t)t * n] = (row == k + t0 + t) ? T(1) : T(0);
        }
        __syncthreads();
        for (int jj = kt - 1; jj >= 0; --jj) {
            const T tw = tau[jj];
            if (tw == T(0)) continue;
            for (int t = wid; t < tw_; t += nwarp) {
                T* E = C + (int64_t)t * n;
                T w = 0;
                for (int r = jj + 1 + lane; r < n; r += 32) w += W[r + (int64_t)jj * n] * E[r];
                w = warp_sum(w) + E[jj];
                const T tww = tw * w;
                for (int r = jj + 1 + lane; r < n; r += 32) E[r] -= tww * W[r + (int64_t)jj * n];
                if (lane == 0) E[jj] -= tww;
            }
            __syncthreads();
        }
        for (int x = tid; x < n * tw_; x += blockDim.x) {
            const int row = x % n, t = t0 + x / n;
            const int dcol = t < keep ? (r_red + k + t) : (t - keep);
            Qs[row + (int64_t)dcol * n] = C[row + (int64_t)(t - t0) * n];
        }
        __syncthreads();
    }
    for (int x = tid; x < n * k; x += blockDim.x) {
        const int row = x % n, col = x / n;
        Qs[row + (int64_t)(r_red + col) * n] = V[row + (int64_t)col * n];
    }
    if (tid == 0) a.kt[i] = kt;
}

// ================================================================== projection
// In-place projection of one 32-wide panel of a block with the box's Q~ (Alg. 2:
// D <- Q~^T D Q~, F <- Q~^T F Q~), as a register-tiled GEMM:
// Alg. 2 projection of box i's block row and column by its completed basis (Sec. 2.1):
//   left  (block in row i):    B[:, c0:c0+32]  <- Q~^T B[:, c0:c0+32]
//   right (block in column i): B[r0:r0+32, :]  <- B[r0:r0+32, :] Q~
// Each thread owns RPT coordinates of the box (a = ty + 32u) times 4 panel lines
// (c = 4 tx + v); Q~ is staged in chunks of 32 rows (coalesced) and the panel is read
// completely into shared memory before anything is written back.
template <class T, int RPT, bool RIGHT>
__global__ void __launch_bounds__(256)
k_proj(LevelArgs<T> a, int cur, const int* __restrict__ w_box, const int* __restrict__ w_blk) {
    constexpr int PW = 32, KC = 32;
    const int w = blockIdx.x;
    const int i = w_box[w], b = w_blk[w];
    const int n = a.n[i];
    const int jb = RIGHT ? a.brow[b] : a.bcol[b];             // the block's other box
    const int nj = a.n[jb];                                   // ... and dimension
    // lines of a box eliminated in an earlier colour are zero except its skeleton part
    // (rectangular fill, Sec. 2.1): only those are projected
    const int p0 = (a.colour[jb] < cur ? nj - a.kt[jb] : 0) + blockIdx.y * PW;
    if (p0 >= nj) return;                                     // panel beyond the block
    const int pw = min(PW, nj - p0);
    const T* __restrict__ Q = a.Q + a.Q_off[i];
    T* B = a.blk + a.blk_off[b];
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nr = (n + KC - 1) / KC * KC;         // n rounded up to whole chunks
    const int lp = nr + 1;                         // padded lines
    T* Ps = reinterpret_cast<T*>(sm_raw);          // panel: PW x lp, Ps[c * lp + q]
    T* Qs = Ps + PW * lp;                          // chunk: KC x lp, Qs[kk * lp + a]
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    // every entry the products read is written (zeros beyond n and beyond the panel)
    if (!RIGHT) {
        for (int x = tid; x < nr * PW; x += 256) {
            const int q = x % nr, c = x / nr;
            Ps[c * lp + q] = (c < pw && q < n) ? B[q + (int64_t)(p0 + c) * n] : T(0);
        }
    } else {
        for (int x = tid; x < nr * PW; x += 256) {
            const int c = x % PW, q = x / PW;
            Ps[c * lp + q] = (c < pw && q < n) ? B[(p0 + c) + (int64_t)q * nj] : T(0);
        }
    }
    T acc[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int k0 = 0; k0 < n; k0 += KC) {
        const int kc = min(KC, n - k0);
        __syncthreads();
        for (int x = tid; x < KC * nr; x += 256) {
            const int kk = x % KC, col = x / KC;
            Qs[kk * lp + col] = (kk < kc && col < n) ? Q[(k0 + kk) + (int64_t)col * n] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            T qv[RPT], pv[4];
            // left: out[a][c] += Q~[q][a] P[q][c];  right: out[c][a] += P[c][q] Q~[q][a]
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int aa = ty + 32 * u;
                qv[u] = aa < n ? Qs[kk * lp + aa] : T(0);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) pv[v] = Ps[(4 * tx + v) * lp + k0 + kk];
#pragma unroll
            for (int u = 0; u < RPT; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += qv[u] * pv[v];
        }
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int aa = ty + 32 * u;
        if (aa >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = 4 * tx + v;
            if (c >= pw) continue;
            if (!RIGHT) B[aa + (int64_t)(p0 + c) * n] = acc[u][v];
            else B[(p0 + c) + (int64_t)aa * nj] = acc[u][v];
        }
    }
}

// ---- the same projection on the tensor cores (float32 factors, boxes <= 128; see
// proj_tc.cuh).  blockIdx.x = box of the colour; its entries pj_ptr[q] .. pj_ptr[q+1]-1
// of `blks` (row i's blocks on the left, their transposes on the right).
template <bool RIGHT>
__global__ void __launch_bounds__(pj::kThreads, 1)
k_proj_tc(LevelArgs<float> a, int cur, const int* __restrict__ boxes, const int* __restrict__ pj_ptr,
          const int* __restrict__ blks, long long budget) {
    using namespace pj;
    extern __shared__ __align__(1024) unsigned char sm_pj[];
    unsigned char* As = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sm_pj) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* ring = As + kABytes;
    Ctrl* ctl = reinterpret_cast<Ctrl*>(ring + (size_t)kStages * kStageBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &ctl->abort;
    const int q = blockIdx.x;
    const int i = boxes[q];
    const int ni = a.n[i];
    const int ks = (ni + BK - 1) / BK;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            tc::mbar_init(&ctl->full[st], kProdWarps);
            tc::mbar_init(&ctl->empty[st], 1);
        }
        for (int x = 0; x < 2; ++x) {
            tc::mbar_init(&ctl->accfull[x], 1);
            tc::mbar_init(&ctl->accempty[x], kEpiWarps);
        }
        for (int x = 0; x < kTrec; ++x) {
            tc::mbar_init(&ctl->tfull[x], 1);
            tc::mbar_init(&ctl->tempty[x], kEpiWarps);
        }
        tc::mbar_init(&ctl->aready, kProdWarps);
        tc::mbar_init(&ctl->drain, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc(&ctl->tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp < kProdWarps) {
        // ---------------- producers
        const int line = tid & 127, h = tid >> 7;
        // Q~^T: A[m][k] = Q~[k][m], K-contiguous; zero beyond n_i
        {
            const float* Q = a.Q + a.Q_off[i];
            for (int sl = 0; sl < ks; ++sl) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = BK * sl + 8 * h + e;
                    v[e] = (line < ni && k < ni) ? Q[k + (int64_t)line * ni] : 0.f;
                }
                unsigned char* d = As + (size_t)sl * 2 * kPart;
                store8(d, d + kPart, tid, v);
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->aready);
        }
        // walk: blocks of the box, 128-line tiles, K slices
        const int e1 = pj_ptr[q + 1];
        int e = pj_ptr[q];
        bool active = false;
        int tn = 0, ntn = 0, sl = 0, nv = 0, nmma = 16, tiles = 0, N = 0, lo = 0, nj = 0;
        int64_t boff = 0;
        auto publish = [&](const TileRec& r) {      // thread 0
            const int slot = tiles % kTrec;
            if (tiles >= kTrec && !*abort) wait_phase(&ctl->tempty[slot], ((tiles / kTrec) - 1) & 1, abort, budget);
            ctl->trec[slot] = r;
            mbar_arrive(&ctl->tfull[slot]);
            ++tiles;
        };
        auto start_tile = [&]() {
            const int n0 = tn * BN;
            nv = min(BN, N - n0);
            nmma = (nv + 15) / 16 * 16;
            sl = 0;
            if (tid == 0) {
                TileRec r;
                if (!RIGHT) { r.C = a.blk + boff + (int64_t)(lo + n0) * ni; r.ls = 1; r.cs = ni; }
                else { r.C = a.blk + boff + lo + n0; r.ls = nj; r.cs = 1; }
                r.mv = ni;
                r.nv = nv;
                r.end = 0;
                r.pad = 0;
                publish(r);
            }
        };
        // next slice: base of its first line and k, strides, header; false when done
        auto next = [&](const float*& base, int64_t& kst, int64_t& lst, int& vlines, int& hdr) -> bool {
            for (;;) {
                if (!active) {
                    if (e >= e1) return false;
                    const int b = blks[e++];
                    const int jb = RIGHT ? a.brow[b] : a.bcol[b];
                    nj = a.n[jb];
                    // lines of a box eliminated in an earlier colour are zero except its
                    // skeleton part (rectangular fill, Sec. 2.1)
                    lo = a.colour[jb] < cur ? nj - a.kt[jb] : 0;
                    N = nj - lo;
                    if (N <= 0) continue;
                    boff = a.blk_off[b];
                    ntn = (N + BN - 1) / BN;
                    tn = 0;
                    start_tile();
                    active = true;
                }
                if (sl < ks) {
                    const int n0 = tn * BN;
                    if (!RIGHT) { base = a.blk + boff + (int64_t)(lo + n0) * ni + BK * sl; kst = 1; lst = ni; }
                    else { base = a.blk + boff + lo + n0 + (int64_t)(BK * sl) * nj; kst = nj; lst = 1; }
                    vlines = nv;
                    hdr = (sl == 0 ? F_FIRST : 0) | (sl == ks - 1 ? F_LAST : 0) | (nmma << 3) | (sl << 12);
                    ++sl;
                    return true;
                }
                if (++tn < ntn) start_tile();
                else active = false;
            }
        };
        auto load = [&](const float* base, int64_t kst, int64_t lst, int vlines, int kmax, float (&v)[8]) {
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int k = 8 * h + x;
                v[x] = (line < vlines && k < kmax) ? base[(int64_t)k * kst + (int64_t)line * lst] : 0.f;
            }
        };
        float rv[kPre][8];
        int hd[kPre];
        bool have[kPre];
#pragma unroll
        for (int j = 0; j < kPre; ++j) { hd[j] = 0; have[j] = false; }
        bool more = true;
        int s = 0;
        auto put = [&](int hdr, const float (&v)[8]) {
            const int st = s % kStages, use = s / kStages;
            ++s;
            if (*abort) return;
            if (use >= 1 && lane == 0) wait_phase(&ctl->empty[st], (use - 1) & 1, abort, budget);
            __syncwarp();
            if (*abort) return;
            unsigned char* d = ring + (size_t)st * kStageBytes;
            store8(d, d + kPart, tid, v);
            if (tid == 0) ctl->hdr[st] = hdr;
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->full[st]);
        };
        bool pending;
        do {
#pragma unroll
            for (int j = 0; j < kPre; ++j) {
                if (have[j]) put(hd[j], rv[j]);
                have[j] = false;
                if (more) {
                    const float* base;
                    int64_t kst, lst;
                    int vlines;
                    more = next(base, kst, lst, vlines, hd[j]);
                    if (more) {
                        const int kmax = ni - BK * ((hd[j] >> 12) & 7);
                        load(base, kst, lst, vlines, kmax, rv[j]);
                        have[j] = true;
                    }
                }
            }
            pending = false;
#pragma unroll
            for (int j = 0; j < kPre; ++j) pending |= have[j];
        } while (more || pending);
        // end markers: a stage for the MMA thread, a tile record for the epilogue
        if (!*abort) {
            const int st = s % kStages, use = s / kStages;
            if (use >= 1 && lane == 0) wait_phase(&ctl->empty[st], (use - 1) & 1, abort, budget);
            __syncwarp();
            if (tid == 0) ctl->hdr[st] = F_END;
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->full[st]);
        }
        if (tid == 0) {
            TileRec r{};
            r.end = 1;
            publish(r);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            bool issued = false;
            if (wait_phase(&ctl->aready, 0, abort, budget)) {
                int s = 0, tile = 0;
                for (;;) {
                    const int st = s % kStages, use = s / kStages;
                    if (!wait_phase(&ctl->full[st], use & 1, abort, budget)) break;
                    const int hdr = ctl->hdr[st];
                    if (hdr & F_END) break;
                    const int acc = tile & 1, accuse = tile >> 1;
                    if ((hdr & F_FIRST) && accuse >= 1 &&
                        !wait_phase(&ctl->accempty[acc], (accuse - 1) & 1, abort, budget))
                        break;
                    tc::fence_after();
                    const uint32_t ab = tc::smem_u32(As + (size_t)((hdr >> 12) & 7) * 2 * kPart);
                    const uint32_t bb = tc::smem_u32(ring + (size_t)st * kStageBytes);
                    const uint32_t d = tmem + (uint32_t)acc * kAccCols;
                    const uint32_t idesc = tc::idesc_tf32(BM, (hdr >> 3) & 0x1ff);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint32_t o = kk * 2 * tc::kLBO;
                        const uint64_t aH = tc::sdesc(ab + o, tc::kLBO, kSBO);
                        const uint64_t aL = tc::sdesc(ab + kPart + o, tc::kLBO, kSBO);
                        const uint64_t bH = tc::sdesc(bb + o, tc::kLBO, kSBO);
                        const uint64_t bL = tc::sdesc(bb + kPart + o, tc::kLBO, kSBO);
                        tc::mma_tf32(d, aL, bH, idesc, ((hdr & F_FIRST) && kk == 0) ? 0 : 1);
                        tc::mma_tf32(d, aH, bL, idesc, 1);
                        tc::mma_tf32(d, aH, bH, idesc, 1);
                    }
                    issued = true;
                    tc::mma_commit(&ctl->empty[st]);
                    if (hdr & F_LAST) {
                        tc::mma_commit(&ctl->accfull[acc]);
                        ++tile;
                    }
                    ++s;
                }
            }
            if (issued) {
                tc::mma_commit(&ctl->drain);
                if (!tc::mbar_wait(&ctl->drain, 0, kWaitCycles)) *abort = 1;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: the tile over the block
        const int qd = warp & 3;
        const int row = 32 * qd + lane;
        int tile = 0;
        for (;;) {
            const int slot = tile % kTrec;
            if (!__all_sync(0xffffffffu, wait_phase(&ctl->tfull[slot], (tile / kTrec) & 1, abort, budget))) break;
            const TileRec r = ctl->trec[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty[slot]);
            if (r.end) break;
            const int acc = tile & 1;
            if (!__all_sync(0xffffffffu, wait_phase(&ctl->accfull[acc], (tile >> 1) & 1, abort, budget))) break;
            tc::fence_after();
            const bool rok = row < r.mv;
            float* Crow = r.C + (int64_t)row * r.ls;
            const uint32_t taddr = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)acc * kAccCols;
            const int ncc = (r.nv + 15) / 16;
            for (int cc = 0; cc < ncc; ++cc) {
                float v[16];
                tc::tmem_ld16(taddr + 16 * cc, v);
                if (rok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = 16 * cc + j;
                        if (col < r.nv) Crow[(int64_t)col * r.cs] = v[j];
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->accempty[acc]);
            ++tile;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (tid == 0 && *abort) dev_fail(a.status, H2_ERR_TIMEOUT, a.level, i);
}

// F truncation after projection (Sec. 2.1: fill is kept in the skeleton coordinates
// only): redundant rows (is_col = 0) or columns (1) of a fill block of box i are
// dropped (set to zero).  Same kernel zeroes the eliminated rows / columns of
// near-field blocks after the Schur update.
template <class T>
__global__ void k_zero_redundant(LevelArgs<T> a, const int* __restrict__ z_box,
                                 const int* __restrict__ z_blk, const int* __restrict__ z_col) {
    const int w = blockIdx.x;
    const int i = z_box[w], b = z_blk[w];
    const int r = a.n[i] - a.kt[i];
    if (r <= 0) return;
    const int rows = a.n[a.brow[b]], cols = a.n[a.bcol[b]];
    T* B = a.blk + a.blk_off[b];
    if (z_col[w] == 0) {
        for (int x = threadIdx.x; x < r * cols; x += blockDim.x) {
            const int rr = x % r, c = x / r;
            B[rr + (int64_t)c * rows] = T(0);
        }
    } else {
        for (int64_t x = threadIdx.x; x < (int64_t)rows * r; x += blockDim.x) B[x] = T(0);
    }
}

// ================================================================== partial LU
// Alg. 2 partial factorisation (Sec. 2.1, Eq. 2.1): LU with partial pivoting of
// D_RR = D_ii[0:r, 0:r] (first maximal |value| wins), P D_RR = L U stored as one r x r
// column-major matrix; the interchanges are replaced in `piv` by the row permutation
// they compose to, (P y)[q] = y[perm[q]].  With `transposed`, DI (offsets of Q) receives
// (L U)^T for the triangular solves of W_L; otherwise DI is scratch here and k_inverse
// fills it with D_RR^-1.
template <class T>
__global__ void __launch_bounds__(256)
k_lu(LevelArgs<T> a, const int* __restrict__ boxes, int in_smem, int transposed) {
    const int i = boxes[blockIdx.x];
    const int n = a.n[i];
    const int r = n - a.kt[i];
    if (r <= 0) return;
    const int tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ T rv[32];
    __shared__ int ri[32];
    __shared__ int piv_s;
    __shared__ T pv_s;
    T* G = a.LU + a.LU_off[i];
    T* W = in_smem ? reinterpret_cast<T*>(sm_raw) : G;
    const T* Dii = a.blk + a.blk_off[a.diag_blk[i]];
    for (int x = tid; x < r * r; x += blockDim.x) {
        const int rr = x % r, c = x / r;
        W[x] = Dii[rr + (int64_t)c * n];
    }
    __syncthreads();
    int* pv = a.piv + a.piv_off[i];
    for (int j = tid; j < r; j += blockDim.x) pv[j] = j;   // defined even if we stop early
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        // argmax |W[a][j]|, a >= j, ties to the lowest index
        T best = T(-1);
        int bi = INT_MAX;
        for (int x = j + tid; x < r; x += blockDim.x) {
            const T v = t_abs(W[x + (int64_t)j * r]);
            if (v > best || (v == best && x < bi)) { best = v; bi = x; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            T bb = T(-1);
            int bx = INT_MAX;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (rv[w] > bb || (rv[w] == bb && ri[w] < bx)) { bb = rv[w]; bx = ri[w]; }
            piv_s = bx;
            pv_s = bb;
        }
        __syncthreads();
        const int p = piv_s;
        // a column without a finite non-zero entry (all NaN leaves bx = INT_MAX) keeps
        // pv[j] = j: the interchanges stored are always valid row indices
        if (!(pv_s > T(0)) || !t_finite(pv_s)) {
            if (tid == 0) dev_fail(a.status, H2_ERR_SINGULAR, a.level, i);
            return;
        }
        if (tid == 0) pv[j] = p;
        if (p != j)
            for (int c = tid; c < r; c += blockDim.x) {
                const T t0 = W[j + (int64_t)c * r];
                W[j + (int64_t)c * r] = W[p + (int64_t)c * r];
                W[p + (int64_t)c * r] = t0;
            }
        __syncthreads();
        const T d = W[j + (int64_t)j * r];
        for (int x = j + 1 + tid; x < r; x += blockDim.x) W[x + (int64_t)j * r] /= d;
        __syncthreads();
        const int m = r - j - 1;
        for (int x = tid; x < m * m; x += blockDim.x) {
            const int rr = j + 1 + x % m, c = j + 1 + x / m;
            W[rr + (int64_t)c * r] -= W[rr + (int64_t)j * r] * W[j + (int64_t)c * r];
        }
        __syncthreads();
    }
    if (in_smem)
        for (int x = tid; x < r * r; x += blockDim.x) G[x] = W[x];
    T* X = a.DI + a.Q_off[i];
    int my[4];                                         // perm[tid + 256 q] (r <= 1024)
    {
        // perm from the interchanges in forward order (temporary: X's last r entries)
        int* sg = reinterpret_cast<int*>(X + (int64_t)r * r - r);
        if (tid == 0) {
            for (int q = 0; q < r; ++q) sg[q] = q;
            for (int j = 0; j < r; ++j) { const int p = pv[j]; const int t0 = sg[j]; sg[j] = sg[p]; sg[p] = t0; }
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) my[q] = (tid + q * 256 < r) ? sg[tid + q * 256] : 0;
        __syncthreads();
        for (int q = 0; q < 4; ++q)
            if (tid + q * 256 < r) pv[tid + q * 256] = my[q];
    }
    if (transposed)                                    // (L U)^T: X[c + q r] = G[q + c r]
        for (int x = tid; x < r * r; x += blockDim.x) X[x / r + (int64_t)(x % r) * r] = W[x];
}

// D_RR^-1 = U^-1 L^-1 P formed column by column from the LU factors of k_lu: column c
// is the triangular solve of P e_c ((P e_c)[q] = 1 where perm[q] = c), 8 columns per warp
// (lu_solve.cuh), the factors staged in shared memory when SM (the first gsz words).
// gridDim.y CTAs per box (blockIdx.x = box of the colour).  The inverse feeds W_U / W_L
// as GEMMs and the diagonal solve step (H2_PREC_TF32X3 by default).
template <class T, int RU, bool SM>
__global__ void __launch_bounds__(256)
k_inverse(LevelArgs<T> a, const int* __restrict__ boxes, int gsz) {
    const int i = boxes[blockIdx.x];
    const int r = a.n[i] - a.kt[i];
    if (r <= 0) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const T* G = a.LU + a.LU_off[i];
    if (SM) {
        T* Gs = reinterpret_cast<T*>(sm_raw);
        for (int x = threadIdx.x; x < r * r && x < gsz; x += blockDim.x) Gs[x] = G[x];
        __syncthreads();
        G = Gs;
    }
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int* perm = a.piv + a.piv_off[i];
    int pq[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
        const int q = lane + 32 * u;
        const int pv = q < r ? perm[q] : -1;
        pq[u] = (unsigned)pv < (unsigned)r ? pv : -1;
    }
    T* X = a.DI + a.Q_off[i];
    for (int c0 = kLuCols * (blockIdx.y * nw + (threadIdx.x >> 5)); c0 < r; c0 += kLuCols * nw * gridDim.y) {
        T x[RU][kLuCols];
#pragma unroll
        for (int c = 0; c < kLuCols; ++c)
#pragma unroll
            for (int u = 0; u < RU; ++u) x[u][c] = pq[u] == c0 + c ? T(1) : T(0);
        lu_solve_warp(x, G, r, lane);
#pragma unroll
        for (int c = 0; c < kLuCols; ++c) {
            if (c0 + c >= r) break;
#pragma unroll
            for (int u = 0; u < RU; ++u)
                if (lane + 32 * u < r) X[lane + 32 * u + (int64_t)(c0 + c) * r] = x[u][c];
        }
    }
}

// Line c (< Nsum_i + kt_i) of the operand of W_U^i / W_L^i: column c of
// [D_{i_R, j} ..., D_{i_R, i_S}] (LEFT, contiguous: ld 1) or row c of
// [D_{j, i_R}; ...; D_{i_S, i_R}] (!LEFT: element q at ptr[q * ld]); null beyond the width.
template <class T, bool LEFT>
__device__ inline void w_line(const LevelArgs<T>& a, int i, int c, const T*& ptr, int64_t& ld) {
    const int n = a.n[i], r = n - a.kt[i], ns = a.Nsum[i];
    ptr = nullptr;
    ld = 0;
    if (c >= ns + a.kt[i]) return;
    if (c >= ns) {
        const T* Dii = a.blk + a.blk_off[a.diag_blk[i]];
        if (LEFT) { ptr = Dii + (int64_t)(r + c - ns) * n; ld = 1; }
        else { ptr = Dii + (r + c - ns); ld = n; }
        return;
    }
    for (int p = a.nb_ptr[i]; p < a.nb_ptr[i + 1]; ++p) {
        const int j = a.nb_col[p];
        if (j != i && a.nbofs[p] <= c && c < a.nbofs[p] + a.n[j]) {
            if (LEFT) { ptr = a.blk + a.blk_off[a.nb_blk[p]] + (int64_t)(c - a.nbofs[p]) * n; ld = 1; }
            else { ptr = a.blk + a.blk_off[a.nb_blkT[p]] + (c - a.nbofs[p]); ld = a.n[j]; }
            return;
        }
    }
}

// The off-diagonal factors of Eq. 2.1 (Sec. 2.1):
// W_U^i = D_RR^-1 [D_{i_R, j} ..., D_{i_R, i_S}]   (LEFT)  and
// W_L^i = [D_{j, i_R}; ...; D_{i_S, i_R}] D_RR^-1  (!LEFT), as 64x64-tiled GEMMs with
// K = r_i; the gathered operand's columns (rows) are located per tile from N(i).
template <class T, bool LEFT>
__global__ void __launch_bounds__(256)
k_wgemm(LevelArgs<T> a, const int* __restrict__ w_box, const int* __restrict__ w_mn) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    __shared__ const T* gptr[64];
    __shared__ int64_t gld[64];
    const int i = w_box[blockIdx.x];
    const int mn = w_mn[blockIdx.x];
    const int n = a.n[i], kt = a.kt[i], r = n - kt, ns = a.Nsum[i];
    const int nt = ns + kt;                       // width of W_U / height of W_L
    const int M = LEFT ? r : nt, N = LEFT ? nt : r;
    const int m0 = (mn >> 16) * BM, n0 = (mn & 0xffff) * BN;
    if (r <= 0 || m0 >= M || n0 >= N) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const T* DI = a.DI + a.Q_off[i];
    // locate the gathered lines: columns of D_{i_R,*} (LEFT) or rows of D_{*,i_R}
    if (tid < 64) w_line<T, LEFT>(a, i, (LEFT ? n0 : m0) + tid, gptr[tid], gld[tid]);
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int k0 = 0; k0 < r; k0 += BK) {
        for (int x = tid; x < BK * BM; x += 256) {
            const int kk = x / BM, rr = x % BM;
            const int gr = m0 + rr, gk = k0 + kk;
            T v = T(0);
            if (gr < M && gk < r) {
                if (LEFT) v = DI[gr + (int64_t)gk * r];
                else if (gptr[rr]) v = gptr[rr][(int64_t)gk * gld[rr]];
            }
            As[kk][rr] = v;
        }
        for (int x = tid; x < BK * BN; x += 256) {
            const int kk = x % BK, cc = x / BK;
            const int gc = n0 + cc, gk = k0 + kk;
            T v = T(0);
            if (gc < N && gk < r) {
                if (LEFT) { if (gptr[cc]) v = gptr[cc][gk]; }
                else v = DI[gk + (int64_t)gc * r];
            }
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = As[kk][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
        __syncthreads();
    }
    T* out = LEFT ? a.WU + a.WU_off[i] : a.WL + a.WL_off[i];
    const int64_t ldo = LEFT ? r : a.WLld[i];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gr = m0 + tx + 16 * u, gc = n0 + ty + 16 * v;
            if (gr < M && gc < N) out[gr + (int64_t)gc * ldo] = acc[u][v];
        }
}

// The same factors by triangular solves with the LU factors (P D_RR = L U), for the
// float32 / float64 factorisations, where D_RR^-1 formed explicitly in the working
// precision would cost refinement steps on ill-conditioned problems:
//   W_U^i = U^-1 L^-1 P [D_{i_R, j} ...]                     (LEFT)
//   W_L^i = [D_{j, i_R}; ...] U^-1 L^-1 P, via W_L^T = P^T L^-T U^-T [...]^T  (!LEFT)
// gridDim.y CTAs per box (blockIdx.x = box of the colour).  Each stages the factors (LU,
// or its transpose for W_L) in shared memory when SM (the first gsz words), and a table
// of the operand's segments (one per neighbour j != i, then i's skeleton part: base,
// line and entry strides, first line, length, prefix of 8-line groups).  Its warps then
// take the 8-line groups in turn (every gridDim.y * 8-th) as the right-hand sides of
// lu_solve.cuh (registers).  RU = ceil(r_max / 32).
template <class T, bool LEFT, int RU, bool SM>
__global__ void __launch_bounds__(256)
k_wtrsm(LevelArgs<T> a, const int* __restrict__ boxes, int gsz) {
    const int i = boxes[blockIdx.x];
    const int n = a.n[i], kt = a.kt[i], r = n - kt, ns = a.Nsum[i];
    if (r <= 0) return;
    const int p0 = a.nb_ptr[i], np = a.nb_ptr[i + 1] - p0;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    unsigned char* tb = sm_raw + ((size_t)gsz * sizeof(T) + 15) / 16 * 16;
    const T** sbase = reinterpret_cast<const T**>(tb);             // np + 1 segments
    int* sofs = reinterpret_cast<int*>(sbase + np + 1);             // first line (column of W_U)
    int* slen = sofs + np + 1;                                       // lines
    int* sls = slen + np + 1;                                        // stride between lines
    int* ses = sls + np + 1;                                         // stride between a line's entries
    int* sgrp = ses + np + 1;                                        // prefix of 8-line groups, np + 2
    for (int t = threadIdx.x; t <= np; t += blockDim.x) {
        if (t < np) {
            const int p = p0 + t, j = a.nb_col[p];
            sbase[t] = a.blk + a.blk_off[LEFT ? a.nb_blk[p] : a.nb_blkT[p]];
            sofs[t] = a.nbofs[p];
            slen[t] = j == i ? 0 : a.n[j];                           // i's own columns: the last segment
            sls[t] = LEFT ? n : 1;
            ses[t] = LEFT ? 1 : a.n[j];
        } else {
            const T* Dii = a.blk + a.blk_off[a.diag_blk[i]];
            sbase[t] = LEFT ? Dii + (int64_t)r * n : Dii + r;
            sofs[t] = ns;
            slen[t] = kt;
            sls[t] = LEFT ? n : 1;
            ses[t] = LEFT ? 1 : n;
        }
    }
    const T* G = LEFT ? a.LU + a.LU_off[i] : a.DI + a.Q_off[i];
    if (SM) {
        T* Gs = reinterpret_cast<T*>(sm_raw);
        for (int x = threadIdx.x; x < r * r; x += blockDim.x) Gs[x] = G[x];
        G = Gs;
    }
    __syncthreads();
    if (threadIdx.x < 32) {                                          // group prefix (warp scan)
        int carry = 0;
        for (int t0 = 0; t0 <= np; t0 += 32) {
            const int t = t0 + threadIdx.x;
            int v = t <= np ? (slen[t] + kLuCols - 1) / kLuCols : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if ((int)threadIdx.x >= o) v += u;
            }
            if (t <= np) sgrp[t + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (threadIdx.x == 0) sgrp[0] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int* perm = a.piv + a.piv_off[i];
    int pq[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {                     // row permutation, bounds-checked
        const int q = lane + 32 * u;
        const int pv = q < r ? perm[q] : 0;
        pq[u] = (unsigned)pv < (unsigned)r ? pv : 0;
    }
    const int64_t ldl = a.WLld[i];
    const int ngrp = sgrp[np + 1];
    for (int g = blockIdx.y * nw + (threadIdx.x >> 5); g < ngrp; g += nw * gridDim.y) {
        int lo = 0, hi = np;                           // last segment with sgrp <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sgrp[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int l0 = (g - sgrp[lo]) * kLuCols;       // first line of the group in the segment
        const int nl = min(kLuCols, slen[lo] - l0);
        const int c0 = sofs[lo] + l0;                  // its column of W_U (row of W_L)
        const T* src0 = sbase[lo] + (int64_t)l0 * sls[lo];
        const int64_t ls = sls[lo], es = ses[lo];
        T x[RU][kLuCols];
#pragma unroll
        for (int c = 0; c < kLuCols; ++c)
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int q = lane + 32 * u;
                x[u][c] = (c < nl && q < r) ? src0[c * ls + (int64_t)(LEFT ? pq[u] : q) * es] : T(0);
            }
        if (LEFT) {
            lu_solve_warp(x, G, r, lane);
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) {
                if (c >= nl) break;
                T* out = a.WU + a.WU_off[i] + (int64_t)(c0 + c) * r;
#pragma unroll
                for (int u = 0; u < RU; ++u)
                    if (lane + 32 * u < r) out[lane + 32 * u] = x[u][c];
            }
        } else {
            lu_solve_t_warp(x, G, r, lane);
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) {
                if (c >= nl) break;
                T* out = a.WL + a.WL_off[i] + (c0 + c);
#pragma unroll
                for (int u = 0; u < RU; ++u)
                    if (lane + 32 * u < r) out[(int64_t)pq[u] * ldl] = x[u][c];
            }
        }
    }
}

// shared memory of k_wtrsm: gsz factor words, then the segment table of up to nbmax + 1
// segments
template <class T>
__host__ __device__ inline size_t wtrsm_smem(int gsz, int nbmax) {
    return ((size_t)gsz * sizeof(T) + 15) / 16 * 16 + (size_t)(nbmax + 1) * (sizeof(void*) + 4 * sizeof(int)) +
           (size_t)(nbmax + 2) * sizeof(int);
}

// ================================================================== Schur update
// Schur complement of Alg. 2 (Sec. 2.1; fill outside the near field goes to F), with
// target-owned accumulation: X_jk -= sum_{i in colour, j,k in N(i)} D_{j,i_R} W_U^i[k]
// as one GEMM per target whose K dimension runs over the contributors.  One CTA per
// target, its 64x64 tiles in turn, 256 threads, 4x4 outputs per thread.
template <class T>
__global__ void __launch_bounds__(256)
k_schur(LevelArgs<T> a, int cur, int tg0, const int* __restrict__ tgt_blk, const int* __restrict__ tgt_ptr,
        const int* __restrict__ c_box, const int* __restrict__ c_ablk, const int* __restrict__ c_kpos) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[2][BK][BM + 1];
    __shared__ T Bs[2][BK][BN + 1];
    const int tt = tg0 + blockIdx.x;              // one CTA per target, its tiles in turn
    const int tb = tgt_blk[tt];
    const int j = a.brow[tb], kb = a.bcol[tb];
    const int nj = a.n[j], nk = a.n[kb];
    // rows / columns of boxes eliminated before (or in) this colour: skeleton part only
    // (their redundant rows and columns are exact zeros: rectangular fill, Sec. 2.1)
    const int row_lo = (a.colour[j] <= cur) ? nj - a.kt[j] : 0;
    const int col_lo = (a.colour[kb] <= cur) ? nk - a.kt[kb] : 0;
    const int m = nj - row_lo, nn = nk - col_lo;
    const int ntm = (m + BM - 1) / BM, ntn = (nn + BN - 1) / BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // this thread's load slots: A rows 4*(tid%16)+q of k-column tid/16; B k-rows 4*(tid%4)+q of column tid/4
    const int la_k = tid >> 4, la_r = 4 * (tid & 15);
    const int lb_c = tid >> 2, lb_k = 4 * (tid & 3);
    for (int tile = 0; tile < ntm * ntn; ++tile) {
        const int m0 = (tile / ntn) * BM, n0 = (tile % ntn) * BN;
        T acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
        // K-steps run over (contributor, 16-wide slice); the next step's operands are
        // fetched into registers while the current step computes from shared memory
        int c = tgt_ptr[tt];
        const int cend = tgt_ptr[tt + 1];
        int k0 = 0, ri = 0;
        const T* A = nullptr;
        const T* B = nullptr;
        auto advance = [&](bool first) -> bool {    // move (c, k0) to the next valid step
            if (!first) {
                k0 += BK;
                if (k0 < ri) return true;
                ++c;
            }
            for (; c < cend; ++c) {
                const int i = c_box[c];
                ri = a.n[i] - a.kt[i];
                if (ri <= 0) continue;
                A = a.blk + a.blk_off[c_ablk[c]] + row_lo;                        // m x ri, ld nj
                // W_U^i holds all n_k columns of a neighbour k (col_lo: skip the zero ones
                // of an eliminated k) but only the skeleton columns of i itself
                B = a.WU + a.WU_off[i] +
                    (int64_t)(a.nbofs[a.nb_ptr[i] + c_kpos[c]] + (kb == i ? 0 : col_lo)) * ri;   // ri x nn, ld ri
                k0 = 0;
                return true;
            }
            return false;
        };
        T ra[4], rb[4];
        auto fetch = [&]() {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gr = m0 + la_r + q, gk = k0 + la_k;
                ra[q] = (gr < m && gk < ri) ? A[gr + (int64_t)gk * nj] : T(0);
                const int gc = n0 + lb_c, gk2 = k0 + lb_k + q;
                rb[q] = (gc < nn && gk2 < ri) ? B[gk2 + (int64_t)gc * ri] : T(0);
            }
        };
        bool have = advance(true);
        if (have) fetch();
        int buf = 0;
        while (have) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[buf][la_k][la_r + q] = ra[q];
                Bs[buf][lb_k + q][lb_c] = rb[q];
            }
            __syncthreads();
            have = advance(false);
            if (have) fetch();                       // overlaps with the products below
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T av[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) av[u] = As[buf][kk][tx + 16 * u];
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = Bs[buf][kk][ty + 16 * v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
            }
            buf ^= 1;                                // the other buffer is free: its last
        }                                            // readers passed this step's barrier
        T* Cm = a.blk + a.blk_off[tb] + row_lo + (int64_t)col_lo * nj;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int gr = m0 + tx + 16 * u, gc = n0 + ty + 16 * v;
                if (gr < m && gc < nn) Cm[gr + (int64_t)gc * nj] -= acc[u][v];
            }
        __syncthreads();                             // the stages are reused by the next tile
    }
}

// ---- tensor-core path: operand packing, records, update (see schur_ws.cuh)

// Live lines of neighbour b of a box of colour `cur`: all n_b of a box eliminated
// later, the skeleton part of one eliminated before (or in) this colour.
template <class T>
__device__ inline int live_lo(const LevelArgs<T>& a, int cur, int b) {
    return a.colour[b] <= cur ? a.n[b] - a.kt[b] : 0;
}

// 16 bytes of hi and lo TF32 parts of four values
__device__ inline void split_store(unsigned char* hi, unsigned char* lo, const float (&x)[4]) {
    float4 h, l;
    h.x = tc::to_tf32(x[0]); l.x = tc::to_tf32(x[0] - h.x);
    h.y = tc::to_tf32(x[1]); l.y = tc::to_tf32(x[1] - h.y);
    h.z = tc::to_tf32(x[2]); l.z = tc::to_tf32(x[2] - h.z);
    h.w = tc::to_tf32(x[3]); l.w = tc::to_tf32(x[3] - h.w);
    *reinterpret_cast<float4*>(hi) = h;
    *reinterpret_cast<float4*>(lo) = l;
}

// Packs one (box i, neighbour position p) pair of the colour (blockIdx.y = 0: A region
// D_{b,i_R}; 1: B region W_U^i[b]) in the layout of schur_ws.cuh.
__global__ void __launch_bounds__(256)
k_schur_pack(LevelArgs<float> a, int cur, const int* __restrict__ pk_box, const int* __restrict__ pk_pos,
             const int64_t* __restrict__ pk_off, unsigned char* __restrict__ pA, unsigned char* __restrict__ pB) {
    const int i = pk_box[blockIdx.x], p = pk_pos[blockIdx.x];
    const int r = a.n[i] - a.kt[i];
    if (r <= 0) return;
    const int b = a.nb_col[p], nb = a.n[b];
    const int G = (nb + 7) / 8;
    const bool isB = blockIdx.y == 1;
    const float* src;
    int64_t ls, ks;                                   // strides of line and k in the source
    int lines;
    if (!isB) {                                       // D_{b,i_R}: block (b, i), live rows of b
        const int lo = live_lo(a, cur, b);
        src = a.blk + a.blk_off[a.nb_blkT[p]] + lo;
        ls = 1;
        ks = nb;
        lines = nb - lo;
    } else {                                          // W_U^i columns of b (ld r)
        const int lo = b == i ? 0 : (a.colour[b] < cur ? nb - a.kt[b] : 0);
        src = a.WU + a.WU_off[i] + (int64_t)(a.nbofs[p] + lo) * r;
        ls = r;
        ks = 1;
        lines = b == i ? a.kt[i] : nb - lo;
    }
    unsigned char* dst = (isB ? pB : pA) + pk_off[p];
    const int gv = (lines + 7) / 8, ns = (r + ws::BK - 1) / ws::BK;
    const int items = ns * 4 * gv * 8;                // (slice, k group, row group, line in group)
    for (int x = threadIdx.x; x < items; x += blockDim.x) {
        const int l8 = x & 7;
        int rest = x >> 3;
        const int g = rest % gv;
        rest /= gv;
        const int q = rest & 3, sl = rest >> 2;
        const int line = 8 * g + l8, k0 = ws::BK * sl + 4 * q;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            v[e] = (line < lines && k0 + e < r) ? __ldg(src + line * ls + (int64_t)(k0 + e) * ks) : 0.f;
        unsigned char* o = dst + (int64_t)sl * 2 * G * ws::kGroup + g * ws::kGroup + q * 128 + l8 * 16;
        split_store(o, o + (int64_t)G * ws::kGroup, v);
    }
}

// Records of one colour's Schur targets and contributors (one thread per record).
// Contributor record e of the tensor-core path: the packed A and B regions.
template <class T>
__device__ inline SchurCon schur_con(const LevelArgs<T>& a, int e, const int* __restrict__ c_box,
                                     const int* __restrict__ c_jpos, const int* __restrict__ c_kpos,
                                     const int64_t* __restrict__ pk_off) {
    const int i = c_box[e];
    const int ri = a.n[i] - a.kt[i];
    SchurCon r;
    r.aoff = pk_off[a.nb_ptr[i] + c_jpos[e]];
    r.boff = pk_off[a.nb_ptr[i] + c_kpos[e]];
    r.ri = ri > 0 ? ri : 0;
    r.pad = 0;
    return r;
}

template <class T>
__global__ void k_schur_prep(LevelArgs<T> a, int cur, int t0, int nt, int e0, int ne,
                             const int* __restrict__ tgt_blk, const int* __restrict__ tgt_ptr,
                             const int* __restrict__ c_box, const int* __restrict__ c_jpos,
                             const int* __restrict__ c_kpos, const int64_t* __restrict__ pk_off,
                             SchurTgt* __restrict__ trec, SchurCon* __restrict__ crec) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < nt) {
        const int tt = t0 + x;
        const int tb = tgt_blk[tt];
        const int j = a.brow[tb], kb = a.bcol[tb];
        const int nj = a.n[j], nk = a.n[kb];
        // a box eliminated in an earlier colour (or the contributor itself) keeps only
        // its skeleton rows / columns: the redundant ones are exact zeros once the box is
        // eliminated, so the update there is zero (rectangular fill, Sec. 2.1)
        const int row_lo = live_lo(a, cur, j);
        const int col_lo = live_lo(a, cur, kb);
        SchurTgt r;
        r.coff = a.blk_off[tb] + row_lo + (int64_t)col_lo * nj;
        r.nj = nj;
        r.m = nj - row_lo;
        r.nn = nk - col_lo;
        r.row_lo = row_lo;
        r.cb = tgt_ptr[tt];
        r.ce = tgt_ptr[tt + 1];
        int nsl = 0;
        for (int e = r.cb; e < r.ce; ++e) {
            const int ri = a.n[c_box[e]] - a.kt[c_box[e]];
            if (ri > 0) nsl += (ri + ws::BK - 1) / ws::BK;
        }
        r.nsl = nsl;
        r.ga = (nj + 7) / 8;
        r.gb = (nk + 7) / 8;
        r.c0 = r.cb < r.ce ? schur_con(a, r.cb, c_box, c_jpos, c_kpos, pk_off) : SchurCon{0, 0, 0, 0};
        trec[tt] = r;
    } else if (x < nt + ne) {
        const int e = e0 + (x - nt);
        crec[e] = schur_con(a, e, c_box, c_jpos, c_kpos, pk_off);
    }
}

// Float32 factor: the same target-owned update on the tcgen05 tensor cores, persistent
// warp-specialised CTAs (two per SM) over the packed operands (schur_ws.cuh); CTA b
// takes targets b, b + gridDim.x, ...; `budget` bounds every pipeline wait (SM cycles).
__global__ void __launch_bounds__(ws::kThreads, ws::kCtasPerSm)
k_schur_tc(LevelArgs<float> a, const SchurTgt* __restrict__ trec, const SchurCon* __restrict__ crec, int ntgt,
           const unsigned char* __restrict__ pA, const unsigned char* __restrict__ pB, long long budget) {
    using namespace ws;
    extern __shared__ __align__(1024) unsigned char sm_tc[];
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sm_tc) + 1023) & ~static_cast<uintptr_t>(1023));
    Ctrl* ctl = reinterpret_cast<Ctrl*>(ring + (size_t)kStages * kStageBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort = &ctl->abort;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            tc::mbar_init(&ctl->full[st], 1);
            tc::mbar_init(&ctl->empty[st], 1);
        }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&ctl->accfull[q], 1);
            tc::mbar_init(&ctl->accempty[q], kEpiWarps);
        }
        for (int q = 0; q < kTrec; ++q) {
            tc::mbar_init(&ctl->tfull[q], 1);
            tc::mbar_init(&ctl->tempty[q], kEpiWarps);
        }
        tc::mbar_init(&ctl->drain, 1);
        *abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tc::tmem_alloc(&ctl->tmem, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = ctl->tmem;

    if (warp == kProdWarp) {
        // ---------------- producer (one thread): bulk copies of packed slices
        if (lane == 0) {
            Walk w{trec, crec, ntgt, a.blk, pA, pB, ctl, budget};
            w.init();
            int s = 0;
            bool copied = false;
            const unsigned char* sa;
            const unsigned char* sb;
            int flags;
            while (w.next(sa, sb, flags)) {
                if (*abort) continue;                                // drain: walk, copy nothing
                const int st = s % kStages, use = s / kStages;
                if (use >= 1 && !wait_phase(&ctl->empty[st], (use - 1) & 1, abort, budget)) continue;
                unsigned char* d = ring + (size_t)st * kStageBytes;
                ctl->hdr[st] = StageHdr{flags, w.nmma};
                mbar_arrive_tx(&ctl->full[st], 2 * (w.abytes + w.bbytes));
                bulk_g2s(d, sa, w.abytes, &ctl->full[st]);
                bulk_g2s(d + kPart, sa + (int64_t)w.tg.ga * kGroup, w.abytes, &ctl->full[st]);
                bulk_g2s(d + 2 * kPart, sb, w.bbytes, &ctl->full[st]);
                bulk_g2s(d + 3 * kPart, sb + (int64_t)w.tg.gb * kGroup, w.bbytes, &ctl->full[st]);
                copied = true;
                ++s;
            }
            // end markers: a stage for the MMA thread, a tile record for the epilogue
            if (!*abort) {
                const int st = s % kStages, use = s / kStages;
                if (use < 1 || wait_phase(&ctl->empty[st], (use - 1) & 1, abort, budget)) {
                    ctl->hdr[st] = StageHdr{F_END, 0};
                    mbar_arrive(&ctl->full[st]);
                }
            }
            TileRec r{};
            r.end = 1;
            w.publish(r);
            // the copies issued have landed before the CTA may exit (full budget): the
            // last stage filled completes once all of them have
            if (copied && *abort) {
                for (int q = 0; q < kStages; ++q) {
                    const int sq = s - 1 - q;
                    if (sq < 0) break;
                    tc::mbar_wait(&ctl->full[sq % kStages], (sq / kStages) & 1, kWaitCycles);
                }
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            int s = 0, tile = 0;
            bool issued = false;
            for (;;) {
                const int st = s % kStages, use = s / kStages;
                if (!wait_phase(&ctl->full[st], use & 1, abort, budget)) break;
                const StageHdr h = ctl->hdr[st];
                if (h.flags & F_END) break;
                const int acc = tile & 1, accuse = tile >> 1;
                if ((h.flags & F_FIRST) && accuse >= 1 &&
                    !wait_phase(&ctl->accempty[acc], (accuse - 1) & 1, abort, budget))
                    break;
                tc::fence_after();
                const uint32_t base = tc::smem_u32(ring + (size_t)st * kStageBytes);
                const uint32_t d = tmem + (uint32_t)acc * kAccCols;
                const uint32_t idesc = tc::idesc_tf32(BM, h.n);
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint32_t o = kk * 2 * tc::kLBO;          // two core matrices per 8 k
                    const uint64_t aH = tc::sdesc(base + o, tc::kLBO, kSBO);
                    const uint64_t aL = tc::sdesc(base + kPart + o, tc::kLBO, kSBO);
                    const uint64_t bH = tc::sdesc(base + 2 * kPart + o, tc::kLBO, kSBO);
                    const uint64_t bL = tc::sdesc(base + 3 * kPart + o, tc::kLBO, kSBO);
                    tc::mma_tf32(d, aL, bH, idesc, ((h.flags & F_FIRST) && kk == 0) ? 0 : 1);   // small terms first
                    tc::mma_tf32(d, aH, bL, idesc, 1);
                    tc::mma_tf32(d, aH, bH, idesc, 1);
                }
                issued = true;
                tc::mma_commit(&ctl->empty[st]);                    // frees the stage
                if (h.flags & F_LAST) {
                    tc::mma_commit(&ctl->accfull[acc]);             // the tile's sum is final
                    ++tile;
                }
                ++s;
            }
            // every MMA issued has completed before tensor memory is freed (full budget)
            if (issued) {
                tc::mma_commit(&ctl->drain);
                if (!tc::mbar_wait(&ctl->drain, 0, kWaitCycles)) *abort = 1;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: C -= accumulator, as reductions in L2
        const int q = warp & 3;                                      // tensor-memory lane quadrant
        const int row = 32 * q + lane;
        int tile = 0;
        // every lane waits, and the warp leaves together if any lane gave up (the
        // warp-wide tcgen05.ld and __syncwarp below need all 32 lanes)
        for (;;) {
            const int slot = tile % kTrec;
            if (!__all_sync(0xffffffffu, wait_phase(&ctl->tfull[slot], (tile / kTrec) & 1, abort, budget))) break;
            const TileRec r = ctl->trec[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty[slot]);
            if (r.end) break;
            const int acc = tile & 1;
            if (!__all_sync(0xffffffffu, wait_phase(&ctl->accfull[acc], (tile >> 1) & 1, abort, budget))) break;
            tc::fence_after();
            const bool rok = row < r.mv;
            float* Crow = r.C + row;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * kAccCols;
            const int ncc = (r.nv + 15) / 16;                        // warp-uniform
            for (int cc = 0; cc < ncc; ++cc) {
                float v[16];
                tc::tmem_ld16(taddr + 16 * cc, v);
                if (rok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = 16 * cc + j;
                        if (col < r.nv) red_add(Crow + (int64_t)col * r.ldc, -v[j]);
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->accempty[acc]);
            ++tile;
        }
    }
    // every role is done (or has given up): free tensor memory
    tc::fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
    if (tid == 0 && *abort) dev_fail(a.status, H2_ERR_TIMEOUT, a.level, -1);
}

// ================================================================== level close
// Parent block (p, q) from its four child pairs: skeleton x skeleton parts of the
// near-field / fill blocks plus the zero-padded couplings S~ (Sec. 2.1, level close).
template <class T>
__global__ void k_close_blocks(LevelArgs<T> a, T* __restrict__ pblk, const int64_t* __restrict__ pblk_off,
                               const int* __restrict__ pbrow, const int* __restrict__ pbcol,
                               const int* __restrict__ cl_dblk, const int* __restrict__ cl_fblk,
                               const int64_t* __restrict__ cl_adm, const double* __restrict__ S,
                               const int64_t* __restrict__ S_off) {
    const int pb = blockIdx.x;
    const int p = pbrow[pb], q = pbcol[pb];
    const int c1 = 2 * p, c2 = 2 * p + 1, e1 = 2 * q, e2 = 2 * q + 1;
    const int kc1 = a.kt[c1], kc2 = a.kt[c2], ke1 = a.kt[e1], ke2 = a.kt[e2];
    const int np = kc1 + kc2, nq = ke1 + ke2;
    T* out = pblk + pblk_off[pb];
    for (int64_t x = threadIdx.x; x < (int64_t)np * nq; x += blockDim.x) {
        const int ar = (int)(x % np), bc = (int)(x / np);
        const int ca = ar < kc1 ? 0 : 1, ea = bc < ke1 ? 0 : 1;
        const int c = ca ? c2 : c1, e = ea ? e2 : e1;
        const int a1 = ca ? ar - kc1 : ar, b1 = ea ? bc - ke1 : bc;
        const int slot = 4 * pb + 2 * ca + ea;
        const int nc = a.n[c], ne = a.n[e];
        const int rc = nc - a.kt[c], re = ne - a.kt[e];
        T v = T(0);
        const int db = cl_dblk[slot];
        if (db >= 0) v += a.blk[a.blk_off[db] + (rc + a1) + (int64_t)(re + b1) * nc];
        const int fb = cl_fblk[slot];
        if (fb >= 0) v += a.blk[a.blk_off[fb] + (rc + a1) + (int64_t)(re + b1) * nc];
        const int64_t ad = cl_adm[slot];
        if (ad >= 0) {
            const int kc = a.k[c], ke = a.k[e];
            if (a1 < kc && b1 < ke) v += (T)S[S_off[ad] + a1 + (int64_t)b1 * kc];
        }
        out[x] = v;
    }
}

// Parent basis V_p = [T~_c1; T~_c2], T~_c = [E_c; 0] (nested basis after projection,
// Sec. 2.1, level close).
template <class T>
__global__ void k_close_basis(LevelArgs<T> a, T* __restrict__ pV, const int64_t* __restrict__ pV_off,
                              const int* __restrict__ pk, const double* __restrict__ E,
                              const int64_t* __restrict__ E_off, int64_t child_first) {
    const int p = blockIdx.x;
    const int c1 = 2 * p, c2 = 2 * p + 1;
    const int kc1 = a.kt[c1], kc2 = a.kt[c2];
    const int np = kc1 + kc2, kp = pk[p];
    T* out = pV + pV_off[p];
    for (int64_t x = threadIdx.x; x < (int64_t)np * kp; x += blockDim.x) {
        const int ar = (int)(x % np), col = (int)(x / np);
        const int c = ar < kc1 ? c1 : c2;
        const int a1 = ar < kc1 ? ar : ar - kc1;
        const int kc = a.k[c];
        T v = T(0);
        if (a1 < kc) v = (T)E[E_off[child_first + c] + a1 + (int64_t)col * kc];
        out[x] = v;
    }
}

// ================================================================== top level
// Dense float64 top matrices of the systems whose top level this is, from the level's
// blocks (blk, working precision) or, at the leaf level, from A's float64 near-field
// blocks (D != nullptr: entry near_entry[b] of D_off).  One thread block per block.
template <class T>
__global__ void k_top_assemble(const int* __restrict__ blist, const T* __restrict__ blk,
                               const int64_t* __restrict__ blk_off, const double* __restrict__ D,
                               const int64_t* __restrict__ D_off, const int64_t* __restrict__ near_entry,
                               const int* __restrict__ brow, const int* __restrict__ bcol,
                               const int* __restrict__ n, const int64_t* __restrict__ ttoff,
                               const int* __restrict__ tsys, const TopSys* __restrict__ tops) {
    const int b = blist[blockIdx.x];
    const int p = brow[b], q = bcol[b];
    const int np = n[p], nq = n[q];
    const TopSys ts = tops[tsys[p]];
    double* dst = ts.A + ttoff[p] + ttoff[q] * ts.nt;
    if (D) {
        const double* src = D + D_off[near_entry[b]];
        for (int64_t x = threadIdx.x; x < (int64_t)np * nq; x += blockDim.x)
            dst[x % np + (x / np) * ts.nt] = src[x];
    } else {
        const T* src = blk + blk_off[b];
        for (int64_t x = threadIdx.x; x < (int64_t)np * nq; x += blockDim.x)
            dst[x % np + (x / np) * ts.nt] = (double)src[x];
    }
}

// Alg. 1, last step: dense LU D_t = L_t U_t of the top level (float64, partial
// pivoting, blocked).
// The top LU runs over all systems at once: panel j0 of every top matrix whose order
// exceeds j0 (blockIdx.x / y / z selects the system, see each kernel).

// Panel factorisation (columns j0..j0+jb of rows j0..nt) with partial pivoting; one
// thread block per system.
__global__ void __launch_bounds__(1024)
k_top_panel(const TopSys* __restrict__ tops, int64_t j0, int nb, DevStatus* st) {
    __shared__ double rv[32];
    __shared__ int64_t ri[32];
    __shared__ int64_t psel;
    __shared__ double pval;
    const TopSys ts = tops[blockIdx.x];
    const int64_t nt = ts.nt;
    if (j0 >= nt) return;
    const int jb = (int)(nt - j0 < nb ? nt - j0 : nb);
    double* A = ts.A;
    int* piv = ts.piv;
    const int tid = threadIdx.x;
    for (int jj = 0; jj < jb; ++jj) {
        const int64_t j = j0 + jj;
        double best = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t x = j + tid; x < nt; x += blockDim.x) {
            const double v = fabs(A[x + j * nt]);
            if (v > best || (v == best && x < bi)) { best = v; bi = x; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int64_t bx = INT64_MAX;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (rv[w] > bb || (rv[w] == bb && ri[w] < bx)) { bb = rv[w]; bx = ri[w]; }
            psel = bx;
            pval = bb;
        }
        __syncthreads();
        if (!(pval > 0.0) || !isfinite(pval)) {              // piv[j] stays unset (checked by its readers)
            if (tid == 0) dev_fail(st, H2_ERR_SINGULAR, -1, (int)j);
            return;
        }
        const int64_t p = psel;
        if (tid == 0) piv[j] = (int)p;
        if (p != j)
            for (int c = tid; c < jb; c += blockDim.x) {
                const double t0 = A[j + (j0 + c) * nt];
                A[j + (j0 + c) * nt] = A[p + (j0 + c) * nt];
                A[p + (j0 + c) * nt] = t0;
            }
        __syncthreads();
        const double d = A[j + j * nt];
        for (int64_t x = j + 1 + tid; x < nt; x += blockDim.x) A[x + j * nt] /= d;
        __syncthreads();
        const int rem = jb - jj - 1;
        const int64_t mrows = nt - j - 1;
        for (int64_t x = tid; x < mrows * rem; x += blockDim.x) {
            const int64_t rr = j + 1 + x % mrows;
            const int64_t c = j + 1 + x / mrows;
            A[rr + c * nt] -= A[rr + j * nt] * A[j + c * nt];
        }
        __syncthreads();
    }
}

// Apply the panel's row interchanges to the columns outside the panel (blockIdx.y =
// system).
__global__ void k_top_swap(const TopSys* __restrict__ tops, int64_t j0, int nb) {
    const TopSys ts = tops[blockIdx.y];
    const int64_t nt = ts.nt;
    if (j0 >= nt) return;
    const int jb = (int)(nt - j0 < nb ? nt - j0 : nb);
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nt || (c >= j0 && c < j0 + jb)) return;
    double* A = ts.A;
    for (int jj = 0; jj < jb; ++jj) {
        const int64_t j = j0 + jj, p = ts.piv[j];
        if (p < j || p >= nt) return;   // panel stopped at a singular pivot (status set)
        if (p != j) {
            const double t0 = A[j + c * nt];
            A[j + c * nt] = A[p + c * nt];
            A[p + c * nt] = t0;
        }
    }
}

// U12 = L11^-1 A12 (unit lower L11 of the panel), one thread per column (blockIdx.y =
// system).
__global__ void k_top_trsm(const TopSys* __restrict__ tops, int64_t j0, int nb) {
    const TopSys ts = tops[blockIdx.y];
    const int64_t nt = ts.nt;
    if (j0 >= nt) return;
    const int jb = (int)(nt - j0 < nb ? nt - j0 : nb);
    const int64_t c = j0 + jb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nt) return;
    const double* A = ts.A;
    double* col = ts.A + c * nt;
    for (int jj = 0; jj < jb; ++jj) {
        const double x = col[j0 + jj];
        for (int r = jj + 1; r < jb; ++r) col[j0 + r] -= A[(j0 + r) + (j0 + jj) * nt] * x;
    }
}

// A22 -= L21 U12 (64x64 tiles, float64; blockIdx.z = system).
__global__ void __launch_bounds__(256)
k_top_gemm(const TopSys* __restrict__ tops, int64_t j0, int nb) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const TopSys ts = tops[blockIdx.z];
    const int64_t nt = ts.nt;
    if (j0 >= nt) return;
    const int jb = (int)(nt - j0 < nb ? nt - j0 : nb);
    const int64_t base = j0 + jb;
    const int64_t m0 = base + (int64_t)blockIdx.x * BM, n0 = base + (int64_t)blockIdx.y * BN;
    if (m0 >= nt || n0 >= nt) return;
    double* A = ts.A;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < jb; k0 += BK) {
        for (int x = tid; x < BK * BM; x += 256) {
            const int kk = x / BM, rr = x % BM;
            const int64_t gr = m0 + rr;
            const int gk = k0 + kk;
            As[kk][rr] = (gr < nt && gk < jb) ? A[gr + (j0 + gk) * nt] : 0.0;
        }
        for (int x = tid; x < BK * BN; x += 256) {
            const int kk = x % BK, cc = x / BK;
            const int64_t gc = n0 + cc;
            const int gk = k0 + kk;
            Bs[kk][cc] = (gc < nt && gk < jb) ? A[(j0 + gk) + gc * nt] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = As[kk][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = Bs[kk][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t gr = m0 + tx + 16 * u, gc = n0 + ty + 16 * v;
            if (gr < nt && gc < nt) A[gr + gc * nt] -= acc[u][v];
        }
}

}  // namespace h2rs
