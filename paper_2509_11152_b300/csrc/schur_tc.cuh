// C -= sum_s A_s B_s for 128 x 64 tiles of C on the tcgen05 tensor cores, with
// float32 operands split into two TF32 parts (a = a_hi + a_lo; the product keeps
// a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in float32 in tensor memory), which
// gives float32-level accuracy at tensor-core rate.
//
// 128 threads.  The K dimension arrives as a sequence of slices of at most 16 k-values
// (each from its own pair of column-major matrices, e.g. one Schur contributor).  Each
// thread keeps the next two slices in registers (fetched two steps ahead, so a global
// load has two tensor-core steps to land), and the shared-memory operand tiles are
// double buffered: an mbarrier per buffer, armed by tcgen05.commit, says when the MMAs
// reading it are done.  48 KB of shared memory and 64 tensor-memory columns per CTA
// let four CTAs share an SM.
#pragma once

#include "tcgen05.cuh"

namespace h2rs {
namespace tc {

constexpr int TBM = 128, TBN = 64, TBK = 16;
constexpr uint32_t kSBO = TBK * 32;                    // bytes per 8-row group
constexpr int kAbytes = TBM * TBK * 4;                 // 8 KB per TF32 part
constexpr int kBbytes = TBN * TBK * 4;                 // 4 KB per TF32 part
constexpr int kStage = 2 * kAbytes + 2 * kBbytes;      // A_hi, A_lo, B_hi, B_lo
constexpr int kSmem = 2 * kStage + 64;                 // two stages + barriers / slot
constexpr uint32_t kTmemCols = 64;                     // fp32 accumulator: 128 lanes x 64
constexpr long long kWaitCycles = 4000000000LL;        // about 2 s at 2 GHz
constexpr int kRA = TBK, kRB = TBN * TBK / 128;        // slice registers per thread

// One K-slice: A (rows of the tile, column-major, lda) and B (k x columns of the tile,
// column-major, ldb), both already offset to the slice's first k; kv <= TBK valid k.
struct Slice {
    const float* A;
    int64_t lda;
    const float* B;
    int64_t ldb;
    int kv;
};

// registers of one thread: A row 32w + lane, TBK/4 k-groups of 4; B sub-tiles
// (8 columns x 16 k) st = w + 4u, 4 k-values each
__device__ inline void load_slice(const Slice& sl, int mv, int nv, float (&ra)[kRA], float (&rb)[kRB]) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int r = 32 * w + l;
#pragma unroll
    for (int kg = 0; kg < TBK / 4; ++kg)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 4 * kg + e;
            ra[4 * kg + e] = (r < mv && k < sl.kv) ? sl.A[r + (int64_t)k * sl.lda] : 0.f;
        }
#pragma unroll
    for (int u = 0; u < kRB / 4; ++u) {
        const int st = w + 4 * u;
        const int col = (st % (TBN / 8)) * 8 + (l & 7);
        const int kg = (st / (TBN / 8)) * 4 + (l >> 3);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 4 * kg + e;
            rb[4 * u + e] = (col < nv && k < sl.kv) ? sl.B[k + (int64_t)col * sl.ldb] : 0.f;
        }
    }
}

__device__ inline void split4(const float* x, float4& hi, float4& lo) {
    hi.x = to_tf32(x[0]); lo.x = to_tf32(x[0] - hi.x);
    hi.y = to_tf32(x[1]); lo.y = to_tf32(x[1] - hi.y);
    hi.z = to_tf32(x[2]); lo.z = to_tf32(x[2] - hi.z);
    hi.w = to_tf32(x[3]); lo.w = to_tf32(x[3] - hi.w);
}

// split into TF32 hi / lo parts and store in the canonical K-major layout (16-byte
// stores; every 8 consecutive lanes fill one 128-byte row of banks)
__device__ inline void store_slice(unsigned char* stage, const float (&ra)[kRA], const float (&rb)[kRB]) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int r = 32 * w + l;
#pragma unroll
    for (int kg = 0; kg < TBK / 4; ++kg) {
        const int off = (r >> 3) * kSBO + kg * 128 + (r & 7) * 16;
        float4 hi, lo;
        split4(ra + 4 * kg, hi, lo);
        *reinterpret_cast<float4*>(stage + off) = hi;
        *reinterpret_cast<float4*>(stage + kAbytes + off) = lo;
    }
#pragma unroll
    for (int u = 0; u < kRB / 4; ++u) {
        const int st = w + 4 * u;
        const int col = (st % (TBN / 8)) * 8 + (l & 7);
        const int kg = (st / (TBN / 8)) * 4 + (l >> 3);
        const int off = (col >> 3) * kSBO + kg * 128 + (col & 7) * 16;
        float4 hi, lo;
        split4(rb + 4 * u, hi, lo);
        *reinterpret_cast<float4*>(stage + 2 * kAbytes + off) = hi;
        *reinterpret_cast<float4*>(stage + 2 * kAbytes + kBbytes + off) = lo;
    }
}

// Epilogue target of a tile: C[0:mv, 0:nv] (column-major, ldc) -= accumulator.
struct TileOut {
    float* C;
    int64_t ldc;
    int mv, nv;
};

// One K-slice plus the tile it belongs to; `first` marks the tile's first slice.
struct SliceT {
    Slice sl;
    TileOut out;
    int first;
};

// Persistent form: the slices of many tiles (produced in order by gen(SliceT&), false
// when there are none left) flow through one tensor-memory accumulator, one pair of
// shared-memory stages and one register prefetch pipeline, so a tile's loads start
// while the previous tile is still being finished.  When a tile's first slice is
// staged, the previous tile's MMAs are waited for and its accumulator is subtracted
// from its C (all 128 threads; row 32w + lane, 64 columns).  Returns false if a
// bounded wait gave up (tiles not yet finished are then left unchanged).
template <class Gen>
__device__ bool tiles_sub(Gen gen, unsigned char* smem) {
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kStage);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kStage + 16);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + 2 * kStage + 20);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        *flag = 0;
    }
    if (w == 0) {
        tmem_alloc(tslot, kTmemCols);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_tf32(TBM, TBN);
    const uint32_t trow = tmem + ((uint32_t)(32 * w) << 16);
    auto epilogue = [&](const TileOut& o) {
        const int r = 32 * w + l;
#pragma unroll
        for (int cc = 0; cc < TBN / 16; ++cc) {
            float v[16];
            tmem_ld16(trow + 16 * cc, v);
            if (r < o.mv)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = 16 * cc + j;
                    if (col < o.nv) o.C[r + (int64_t)col * o.ldc] -= v[j];
                }
        }
    };
    SliceT t0, t1;
    float ra0[kRA], rb0[kRB], ra1[kRA], rb1[kRB];
    bool have0 = gen(t0);
    if (have0) load_slice(t0.sl, t0.out.mv, t0.out.nv, ra0, rb0);
    bool have1 = have0 && gen(t1);
    if (have1) load_slice(t1.sl, t1.out.mv, t1.out.nv, ra1, rb1);
    int s = 0;
    bool acc_valid = false;
    TileOut acc{};
    auto step = [&](SliceT& t, float (&ra)[kRA], float (&rb)[kRB], bool& have) -> bool {
        if (!have) return false;
        const int buf = s & 1;
        int late = 0;
        if (t.first && acc_valid) {
            // finish the previous tile: all its MMAs (up to step s-1) must be complete
            if (!mbar_wait(&mbar[(s - 1) & 1], ((s - 1) >> 1) & 1, kWaitCycles)) late = 1;
            if (!__syncthreads_or(late)) {
                fence_after();
                epilogue(acc);
                fence_before();
            } else {
                late = 1;
            }
        } else if (s >= 2 && !mbar_wait(&mbar[buf], ((s >> 1) - 1) & 1, kWaitCycles)) {
            late = 1;
        }
        if (!late) store_slice(smem + buf * kStage, ra, rb);
        fence_proxy_async();
        if (__syncthreads_or(late)) {
            if (tid == 0) *flag = 1;
            return false;
        }
        const int first = t.first;
        if (first) { acc = t.out; acc_valid = true; }
        if (tid == 0) {                                  // the MMAs first: gen may wait on loads
            fence_after();
            const uint32_t base = smem_u32(smem + buf * kStage);
#pragma unroll
            for (int kk = 0; kk < TBK / 8; ++kk) {
                const uint32_t o = kk * 2 * kLBO;          // two core matrices per 8 k-values
                const uint64_t aH = sdesc(base + o, kLBO, kSBO), aL = sdesc(base + kAbytes + o, kLBO, kSBO);
                const uint64_t bH = sdesc(base + 2 * kAbytes + o, kLBO, kSBO);
                const uint64_t bL = sdesc(base + 2 * kAbytes + kBbytes + o, kLBO, kSBO);
                mma_tf32(tmem, aL, bH, idesc, (first && kk == 0) ? 0 : 1);   // small terms first
                mma_tf32(tmem, aH, bL, idesc, 1);
                mma_tf32(tmem, aH, bH, idesc, 1);
            }
            mma_commit(&mbar[buf]);
        }
        have = gen(t);                                   // the slice two steps ahead
        if (have) load_slice(t.sl, t.out.mv, t.out.nv, ra, rb);
        ++s;
        return true;
    };
    while (step(t0, ra0, rb0, have0) && step(t1, ra1, rb1, have1)) {
    }
    // the last tile: wait for every MMA issued, then finish it
    if (s > 0 && tid == 0 && !mbar_wait(&mbar[(s - 1) & 1], ((s - 1) >> 1) & 1, kWaitCycles)) *flag = 1;
    __syncthreads();
    const bool ok = *flag == 0;
    if (ok && acc_valid) {
        fence_after();
        epilogue(acc);
    }
    fence_before();
    __syncthreads();
    if (w == 0) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    return ok;
}

}  // namespace tc
}  // namespace h2rs
