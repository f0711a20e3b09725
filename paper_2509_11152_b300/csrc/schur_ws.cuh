// Target-owned Schur update X_jk -= sum_i D_{j,i_R} W_U^i[k] of one colour (Alg. 2,
// Sec. 2.1 step 3) on the tcgen05 tensor cores, with float32 operands split into two
// TF32 parts (a = a_hi + a_lo; the product keeps a_hi b_hi + a_hi b_lo + a_lo b_hi,
// accumulated in float32 in tensor memory): float32-level accuracy at tensor rate.
//
// Operand packing.  Before the update, every operand of the colour is split once and
// laid out for the tensor cores (k_schur_pack): for each box i of the colour and each
// neighbour position p (box b = N(i)[p]), the A region holds D_{b,i_R} (the live rows
// of b: its skeleton rows once b is eliminated) and the B region holds the columns of
// W_U^i that belong to b (its live columns), both as 16-wide K slices of TF32 hi and lo
// parts in the no-swizzle K-major core-matrix layout of tcgen05.cuh:
//   element (line, k) of slice s = k / 16 sits at byte
//     s * 2G*512 + part * G*512 + (line / 8) * 512 + ((k % 16) / 4) * 128
//       + (line % 8) * 16 + (k % 4) * 4,      G = ceil(n_b / 8), part 0 hi, 1 lo,
// zero beyond the live lines (up to a multiple of 8) and beyond r_i (up to a multiple
// of 16).  A 128-line tile of one slice is then one contiguous run of whole 512-byte
// row groups, copied into a shared-memory stage with one bulk copy per part.  A region
// is shared by every target its operand feeds (about C_sp of them); region offsets are
// bounded by n_b and n_i, so the host places them before the ranks are known.
//
// Update: two persistent CTAs per SM (each holding half of the SM's tensor memory and
// of its shared memory, so that one CTA's record-fetch stalls overlap the other's
// work), warp-specialised:
//  - warp 0 lane 0 (producer) walks this CTA's targets (every gridDim.x-th of the
//    colour, the records of the next two loaded while the current one is sliced), their
//    128 x 128 tiles and, per tile, the K slices of its contributors: per slice it
//    waits for a free stage, announces the byte count on the stage's mbarrier and
//    issues four bulk copies (A hi / lo, B hi / lo) that complete on it;
//  - warp 1 lane 0 issues the MMAs into one of two tensor-memory accumulators of 128
//    columns, so a tile's MMAs overlap the previous tile's epilogue;
//  - warps 2-5 (epilogue, one per 32-lane quadrant of tensor memory) read the
//    finished accumulator and subtract it from C with fire-and-forget reductions in
//    L2 (red.global.add of -acc: no read round trip on the SM; every entry of C is
//    updated by one tile of one launch, so the result is that of C - acc).
// Hand-offs are mbarriers: stage full (transaction count) / empty, accumulator full /
// empty, tile record full / empty.  Every wait is bounded (`budget` SM cycles); a wait
// that runs out raises the CTA's abort flag, after which the producer finishes its walk
// without copying, the other roles leave their loops, the producer waits (full budget)
// for the copies it issued, the MMA thread for its MMAs, and tensor memory is freed.
#pragma once

#include "factor_args.cuh"
#include "tcgen05.cuh"

namespace h2rs {
namespace ws {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int kStages = 3;
constexpr int kCtasPerSm = 2;                      // two independent pipelines per SM
constexpr int kProdWarp = 0, kMmaWarp = 1, kEpi0 = 2, kEpiWarps = 4;
constexpr int kThreads = 32 * (kEpi0 + kEpiWarps);   // 192
constexpr uint32_t kGroup = 512;                   // bytes of 8 lines x 16 k (one row group)
constexpr uint32_t kSBO = kGroup;                  // next 8-line group (K-major, 16 k)
constexpr int kPart = BM / 8 * kGroup;             // 8 KB: one TF32 part of a 128-line tile
constexpr int kStageBytes = 4 * kPart;             // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kAccCols = BN;                  // float32 accumulator columns per tile
constexpr uint32_t kTmemCols = 2 * kAccCols;       // two accumulators
constexpr int kTrec = 4;                           // tile-record ring
constexpr long long kWaitCycles = 4000000000LL;    // about 2 s at 2 GHz

enum { F_FIRST = 1, F_LAST = 2, F_END = 4 };

// bytes of the packed region of one (box i, neighbour b) pair: ceil(n_i / 16) slices of
// two parts of ceil(n_b / 8) row groups
__host__ __device__ inline int64_t pack_region_bytes(int n_i, int n_b) {
    return (int64_t)((n_i + BK - 1) / BK) * 2 * ((n_b + 7) / 8) * kGroup;
}

struct StageHdr {
    int flags;
    int n;                                         // MMA N of the tile (multiple of 16)
};
struct TileRec {
    float* C;                                      // C[0:mv, 0:nv], column-major, ld ldc
    int64_t ldc;
    int mv, nv;
    int end;
    int pad;
};
struct Ctrl {
    uint64_t full[kStages], empty[kStages];
    uint64_t accfull[2], accempty[2];
    uint64_t tfull[kTrec], tempty[kTrec];
    uint64_t drain;
    StageHdr hdr[kStages];
    TileRec trec[kTrec];
    uint32_t tmem;
    int abort;                                     // accessed through volatile pointers
};
constexpr int kSmem = kStages * kStageBytes + (int)sizeof(Ctrl) + 1024;   // + alignment slack

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(bar)) : "memory");
}
// arrive and raise the phase's expected transaction count by `bytes`
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) that
// completes `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(tc::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar)) : "memory");
}

// C[p] += v in L2 (no value returned)
__device__ __forceinline__ void red_add(float* p, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" :: "l"(p), "f"(v) : "memory");
}

// waits for the phase of the given parity; false (and the abort flag raised) when the
// budget runs out, false at once when another role has aborted
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort,
                                           long long budget) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > budget) {
            *abort = 1;
            return false;
        }
    }
}

// Producer walk over this CTA's targets, their tiles, contributors and K slices.
struct Walk {
    const SchurTgt* __restrict__ trec;
    const SchurCon* __restrict__ crec;
    int ntgt;
    float* blk;
    const unsigned char* pA;                       // packed A / B regions of the colour
    const unsigned char* pB;
    Ctrl* ctl;
    long long budget;
    int tnext = 0;                                 // the next target (>= ntgt: none)
    SchurTgt nx{}, nx2{};                          // records of the next two targets
    bool active = false;
    SchurTgt tg{};
    SchurCon cr{}, cn{};                           // current contributor, the next one
    int c = 0, s = 0, tm = 0, tn = 0, ntm = 0, ntn = 0, sl = 0, nmma = 16;
    int tiles = 0;                                 // tile records published
    uint32_t abytes = 0, bbytes = 0;               // bytes of one part of the tile's slices

    __device__ __forceinline__ void init() {
        tnext = blockIdx.x;
        if (tnext < ntgt) nx = trec[tnext];
        if (tnext + (int)gridDim.x < ntgt) nx2 = trec[tnext + gridDim.x];
    }

    __device__ __forceinline__ void publish(const TileRec& r) {
        const int slot = tiles % kTrec;
        volatile int* ab = &ctl->abort;
        if (tiles >= kTrec && !*ab) wait_phase(&ctl->tempty[slot], ((tiles / kTrec) - 1) & 1, ab, budget);
        ctl->trec[slot] = r;
        mbar_arrive(&ctl->tfull[slot]);
        ++tiles;
    }

    __device__ __forceinline__ void start_tile() {
        const int m0 = tm * BM, n0 = tn * BN;
        const int mv = min(BM, tg.m - m0), nv = min(BN, tg.nn - n0);
        nmma = (nv + 15) / 16 * 16;
        abytes = (uint32_t)((mv + 7) / 8) * kGroup;
        bbytes = (uint32_t)((nv + 7) / 8) * kGroup;
        c = tg.cb;
        s = 0;
        sl = 0;
        cr = tg.c0;
        if (c + 1 < tg.ce) cn = crec[c + 1];
        TileRec r;
        r.C = blk + tg.coff + m0 + (int64_t)n0 * tg.nj;
        r.ldc = tg.nj;
        r.mv = mv;
        r.nv = nv;
        r.end = 0;
        r.pad = 0;
        publish(r);
    }

    // next slice: operand sources of its four parts and its header; false when done
    __device__ __forceinline__ bool next(const unsigned char*& a, const unsigned char*& b, int& flags) {
        for (;;) {
            if (!active) {
                if (tnext >= ntgt) return false;
                tg = nx;
                nx = nx2;
                tnext += gridDim.x;
                if (tnext + (int)gridDim.x < ntgt) nx2 = trec[tnext + gridDim.x];   // two targets ahead
                ntm = (tg.m + BM - 1) / BM;
                ntn = (tg.nn + BN - 1) / BN;
                if (ntm <= 0 || ntn <= 0 || tg.nsl == 0) continue;   // nothing to subtract
                tm = tn = 0;
                start_tile();
                active = true;
            }
            while (c < tg.ce) {
                if (s * BK < cr.ri) {
                    a = pA + cr.aoff + (int64_t)s * 2 * tg.ga * kGroup + (int64_t)tm * (BM / 8) * kGroup;
                    b = pB + cr.boff + (int64_t)s * 2 * tg.gb * kGroup + (int64_t)tn * (BN / 8) * kGroup;
                    flags = (sl == 0 ? F_FIRST : 0) | (sl == tg.nsl - 1 ? F_LAST : 0);
                    ++sl;
                    ++s;
                    return true;
                }
                if (++c < tg.ce) {
                    cr = cn;
                    if (c + 1 < tg.ce) cn = crec[c + 1];
                }
                s = 0;
            }
            if (++tn == ntn) { tn = 0; ++tm; }
            if (tm < ntm) start_tile();
            else active = false;
        }
    }
};

}  // namespace ws
}  // namespace h2rs
