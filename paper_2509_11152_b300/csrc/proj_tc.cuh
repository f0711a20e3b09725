// Projection of a box's block row or block column by its completed basis (Alg. 2:
// D <- Q~^T D Q~, F <- Q~^T F Q~; Sec. 2.1 step 2) on the tcgen05 tensor cores, float32
// operands split into two TF32 parts (hi*hi + hi*lo + lo*hi, float32 accumulation in
// tensor memory), for boxes of at most 128 points.
//
// Both sides are the product C = Q~^T B with Q~^T as the MMA's A operand:
//   left  (block (i, j) of row i):    B = the block,   C overwrites the block;
//   right (block (j, i) of column i): B = the block^T, C^T overwrites the block,
// where only the live lines of j take part (all of them, or the skeleton part once j
// is eliminated: its other lines are zero).  One CTA per box of the colour, one launch
// per side (two boxes of a colour may share a fill block, one from each side):
//  - warps 0-7 (producers) first store Q~^T, split, as kKS K slices of 128 rows in the
//    no-swizzle K-major layout of tcgen05.cuh (the block's 16-wide K slices then pair
//    with a fixed A slice), then walk the box's blocks and their 128-line tiles, loading
//    each 16-wide K slice of B into registers (plain loads in the
//    block's own order, K-contiguous on the left, line-contiguous on the right)
//    kPre slices ahead of its use, splitting it and storing it into a kStages-deep ring;
//  - warp 8 lane 0 issues the MMAs into one of two 128-column accumulators;
//  - warps 9-12 (one per 32-lane quadrant of tensor memory) write the finished tile
//    back over the block (each block is read by its own tile before it is written, and
//    different tiles of a block cover different lines).
// Every wait is bounded as in schur_ws.cuh; the producers keep walking without storing
// once a wait has given up, and the MMA thread waits for its MMAs before tensor memory
// is freed.
#pragma once

#include "factor_args.cuh"
#include "tcgen05.cuh"

namespace h2rs {
namespace pj {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int kKS = BM / BK;                       // K slices of Q~^T (n_i <= 128)
constexpr int kStages = 5;
constexpr int kPre = 6;                            // slices held in producer registers
constexpr int kProdWarps = 8, kMmaWarp = 8, kEpi0 = 9, kEpiWarps = 4;
constexpr int kThreads = 32 * (kProdWarps + 1 + kEpiWarps);   // 416 (128 registers each)
constexpr uint32_t kSBO = BK * 32;                 // 512 bytes per 8-line group
constexpr int kPart = BM * BK * 4;                 // 8 KB: one TF32 part of a 128-line slice
constexpr int kABytes = kKS * 2 * kPart;           // Q~^T, hi and lo of every slice
constexpr int kStageBytes = 2 * kPart;             // B hi, B lo
constexpr uint32_t kAccCols = BN;
constexpr uint32_t kTmemCols = 2 * kAccCols;
constexpr int kTrec = 4;
constexpr long long kWaitCycles = 4000000000LL;

enum { F_FIRST = 1, F_LAST = 2, F_END = 4 };

struct TileRec {
    float* C;                                      // element (m, n') at C + m * ls + n' * cs
    int64_t ls, cs;
    int mv, nv;
    int end;
    int pad;
};
struct Ctrl {
    uint64_t full[kStages], empty[kStages];
    uint64_t accfull[2], accempty[2];
    uint64_t tfull[kTrec], tempty[kTrec];
    uint64_t aready, drain;
    int hdr[kStages];                              // flags | n << 3 | slice << 12
    TileRec trec[kTrec];
    uint32_t tmem;
    int abort;                                     // accessed through volatile pointers
};
constexpr int kSmem = kABytes + kStages * kStageBytes + (int)sizeof(Ctrl) + 1024;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort, long long budget) {
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

// hi / lo TF32 parts of 8 consecutive k of one line into a K-major slice pair
// (line = thread & 127, k half = thread >> 7)
__device__ __forceinline__ void store8(unsigned char* hi, unsigned char* lo, int tid, const float (&v)[8]) {
    const int line = tid & 127, h = tid >> 7;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int off = (line >> 3) * kSBO + (2 * h + g) * 128 + (line & 7) * 16;
        float4 a, b;
        a.x = tc::to_tf32(v[4 * g + 0]); b.x = tc::to_tf32(v[4 * g + 0] - a.x);
        a.y = tc::to_tf32(v[4 * g + 1]); b.y = tc::to_tf32(v[4 * g + 1] - a.y);
        a.z = tc::to_tf32(v[4 * g + 2]); b.z = tc::to_tf32(v[4 * g + 2] - a.z);
        a.w = tc::to_tf32(v[4 * g + 3]); b.w = tc::to_tf32(v[4 * g + 3] - a.w);
        *reinterpret_cast<float4*>(hi + off) = a;
        *reinterpret_cast<float4*>(lo + off) = b;
    }
}

}  // namespace pj
}  // namespace h2rs
