// Triangular solves of one warp with the partial-LU factors of a redundant block
// (Sec. 2.1, Eq. 2.1: P D_RR = L U, L unit lower, U upper, stored as one r x r
// column-major matrix G of storage type T), for kLuCols right-hand sides of type V held
// in registers: row q of right-hand side c is x[q / 32][c] of lane q % 32, rows q >= r
// are zero and stay zero; the arithmetic is in V.
// Column j of the eliminated factor is read by the lanes in one coalesced load (G may sit
// in global or shared memory: generic loads) and the pivot row's value is broadcast by
// a shuffle, so the warp needs no barrier; RU = ceil(r / 32) row registers per
// right-hand side (r <= 32 RU).
#pragma once

#include <cstdint>

namespace h2rs {

constexpr int kLuCols = 8;

// x <- U^-1 L^-1 x, G column-major (L below the diagonal, U on and above it)
template <class V, class T, int RU>
__device__ __forceinline__ void lu_solve_warp(V (&x)[RU][kLuCols], const T* G, int r, int lane) {
#pragma unroll
    for (int jb = 0; jb < RU; ++jb) {                     // L: forward, unit diagonal
        const int jend = min(32, r - 32 * jb);
        for (int jl = 0; jl < jend; ++jl) {
            const int j = 32 * jb + jl;
            const T* gc = G + (int64_t)j * r;
            V xj[kLuCols];
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) xj[c] = __shfl_sync(0xffffffffu, x[jb][c], jl);
#pragma unroll
            for (int u = jb; u < RU; ++u) {
                const int q = lane + 32 * u;
                const V l = (q > j && q < r) ? (V)gc[q] : V(0);
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[u][c] -= l * xj[c];
            }
        }
    }
#pragma unroll
    for (int jb = RU - 1; jb >= 0; --jb) {                // U: backward
        const int jend = min(32, r - 32 * jb);
        for (int jl = jend - 1; jl >= 0; --jl) {
            const int j = 32 * jb + jl;
            const T* gc = G + (int64_t)j * r;
            const V inv = V(1) / (V)gc[j];
            V xj[kLuCols];
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) xj[c] = __shfl_sync(0xffffffffu, x[jb][c], jl) * inv;
            if (lane == jl) {
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[jb][c] = xj[c];
            }
#pragma unroll
            for (int u = 0; u <= jb; ++u) {
                const int q = lane + 32 * u;
                const V v = (q < j) ? (V)gc[q] : V(0);
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[u][c] -= v * xj[c];
            }
        }
    }
}

// x <- L^-T U^-T x with Gt = G^T (column j of Gt is row j of G: U^T's column j on and
// below the diagonal, L^T's column j above it)
template <class V, class T, int RU>
__device__ __forceinline__ void lu_solve_t_warp(V (&x)[RU][kLuCols], const T* Gt, int r, int lane) {
#pragma unroll
    for (int jb = 0; jb < RU; ++jb) {                     // U^T: forward, diagonal U_jj
        const int jend = min(32, r - 32 * jb);
        for (int jl = 0; jl < jend; ++jl) {
            const int j = 32 * jb + jl;
            const T* gc = Gt + (int64_t)j * r;
            const V inv = V(1) / (V)gc[j];
            V xj[kLuCols];
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) xj[c] = __shfl_sync(0xffffffffu, x[jb][c], jl) * inv;
            if (lane == jl) {
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[jb][c] = xj[c];
            }
#pragma unroll
            for (int u = jb; u < RU; ++u) {
                const int q = lane + 32 * u;
                const V v = (q > j && q < r) ? (V)gc[q] : V(0);
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[u][c] -= v * xj[c];
            }
        }
    }
#pragma unroll
    for (int jb = RU - 1; jb >= 0; --jb) {                // L^T: backward, unit diagonal
        const int jend = min(32, r - 32 * jb);
        for (int jl = jend - 1; jl >= 0; --jl) {
            const int j = 32 * jb + jl;
            const T* gc = Gt + (int64_t)j * r;
            V xj[kLuCols];
#pragma unroll
            for (int c = 0; c < kLuCols; ++c) xj[c] = __shfl_sync(0xffffffffu, x[jb][c], jl);
#pragma unroll
            for (int u = 0; u <= jb; ++u) {
                const int q = lane + 32 * u;
                const V l = (q < j) ? (V)gc[q] : V(0);
#pragma unroll
                for (int c = 0; c < kLuCols; ++c) x[u][c] -= l * xj[c];
            }
        }
    }
}

}  // namespace h2rs
