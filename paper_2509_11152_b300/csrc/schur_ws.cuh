// Target-owned Schur update X_jk -= sum_i D_{j,i_R} W_U^i[k] of one colour (Alg. 2,
// Sec. 2.1 step 3) on the tcgen05 tensor cores, with float32 operands split into two
// TF32 parts (a = a_hi + a_lo; the product keeps a_hi b_hi + a_hi b_lo + a_lo b_hi,
// accumulated in float32 in tensor memory): float32-level accuracy at tensor rate.
//
// One persistent CTA per SM, warp-specialised:
//  - warps 0-7 (producers) take targets from a global counter, walk each target's
//    128 x 128 tiles and, per tile, the 16-wide K slices of its contributors.  Each
//    slice is loaded into registers kPrefetch slices ahead of its use (plain global
//    loads, no alignment needed: blocks sit at arbitrary offsets of the arena), split
//    into TF32 hi / lo parts and stored into a kStages-deep ring of shared-memory
//    stages in the no-swizzle K-major layout of tcgen05.cuh;
//  - warp 8 issues the MMAs (one thread) into one of two tensor-memory accumulators
//    of 128 columns, so a tile's MMAs overlap the previous tile's epilogue;
//  - warps 9-12 (epilogue, one per 32-lane quadrant of tensor memory) copy C of
//    their next tile into shared memory (cp.async) as soon as its record is
//    published, then wait for its accumulator and write C - acc back (each thread
//    owns one row of the tile, so it reads only what it copied itself).
// Hand-offs are mbarriers: stage full / empty, accumulator full / empty, tile record
// full / empty.  Every wait is bounded (`budget` SM cycles); a wait that runs out
// raises the CTA's abort flag, after which the producers drain the target counter
// without waiting or storing, the other roles leave their loops, the MMA thread waits
// (with the full budget) for its own MMAs, and tensor memory is freed.
#pragma once

#include "factor_args.cuh"
#include "tcgen05.cuh"

namespace h2rs {
namespace ws {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int kStages = 5;
constexpr int kPrefetch = 3;                       // slices held in producer registers
constexpr int kProdWarps = 8, kEpiWarps = 4;
constexpr int kProd = 32 * kProdWarps;             // 256 producer threads
constexpr int kMmaWarp = kProdWarps;               // warp 8
constexpr int kEpi0 = kProdWarps + 1;              // first epilogue warp
constexpr int kThreads = 32 * (kProdWarps + 1 + kEpiWarps);   // 416: at most 4 warps per
                                                   // SM sub-partition, 128 registers each
constexpr uint32_t kSBO = BK * 32;                 // bytes per 8-row group (K-major, 16 k)
constexpr int kPart = BM * BK * 4;                 // 8 KB: one TF32 part of a 128-line operand
constexpr int kStageBytes = 4 * kPart;             // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kAccCols = BN;                  // float32 accumulator columns per tile
constexpr uint32_t kTmemCols = 2 * kAccCols;       // two accumulators
constexpr int kTrec = 4;                           // tile-record ring
constexpr long long kWaitCycles = 4000000000LL;    // about 2 s at 2 GHz

enum { F_FIRST = 1, F_LAST = 2, F_END = 4 };

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
    int next_tgt;
    int abort;                                     // accessed through volatile pointers
};
constexpr int kCBytes = BM * BN * 4;               // C tile staged by the epilogue (ld BM)
constexpr int kSmem = kStages * kStageBytes + kCBytes + (int)sizeof(Ctrl) + 1024;   // + alignment slack

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ inline void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_u32(bar)) : "memory");
}

// waits for the phase of the given parity; false (and the abort flag raised) when the
// budget runs out, false at once when another role has aborted
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

__device__ inline void prod_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// One K slice as the producers see it: where its operands start and which tile it
// belongs to.  Identical in every producer thread.
struct SliceMeta {
    const float* A;                                // rows of the tile, column-major (lda)
    const float* B;                                // columns of the tile, k contiguous (ldb)
    int64_t lda, ldb;
    int kv, mv, nv;                                // valid k, rows, columns
    int flags, n;
};

// Producer-side walk over targets, tiles, contributors and K slices (all producer
// threads execute it in step; the target index is fetched by thread 0 and broadcast).
struct Walk {
    const SchurTgt* __restrict__ trec;
    const SchurCon* __restrict__ crec;
    int ntgt;
    int* counter;
    float* blk;
    const float* WU;
    Ctrl* ctl;
    int tid;
    long long budget;
    bool active = false;
    SchurTgt tg{};
    SchurCon cr{};
    int c = 0, k0 = 0, tm = 0, tn = 0, ntm = 0, ntn = 0, nsl = 0, sl = 0, nmma = 16;
    int tiles = 0;                                 // tile records published
    int mv = 0, nv = 0;

    __device__ __forceinline__ void publish(const TileRec& r) {    // thread 0 only
        const int slot = tiles % kTrec;
        volatile int* ab = &ctl->abort;
        if (tiles >= kTrec && !*ab) wait_phase(&ctl->tempty[slot], ((tiles / kTrec) - 1) & 1, ab, budget);
        ctl->trec[slot] = r;
        mbar_arrive(&ctl->tfull[slot]);
        ++tiles;
    }

    __device__ __forceinline__ void start_tile() {
        const int m0 = tm * BM, n0 = tn * BN;
        mv = min(BM, tg.m - m0);
        nv = min(BN, tg.nn - n0);
        nmma = (nv + 15) / 16 * 16;
        c = tg.cb;
        k0 = 0;
        sl = 0;
        cr = crec[c];
        if (tid == 0) {
            TileRec r;
            r.C = blk + tg.coff + m0 + (int64_t)n0 * tg.nj;
            r.ldc = tg.nj;
            r.mv = mv;
            r.nv = nv;
            r.end = 0;
            r.pad = 0;
            publish(r);
        }
    }

    // next slice, false when the counter is exhausted
    __device__ __forceinline__ bool next(SliceMeta& m) {
        for (;;) {
            if (!active) {
                prod_sync();
                if (tid == 0) ctl->next_tgt = atomicAdd(counter, 1);
                prod_sync();
                const int t = ctl->next_tgt;
                if (t >= ntgt) return false;
                tg = trec[t];
                ntm = (tg.m + BM - 1) / BM;
                ntn = (tg.nn + BN - 1) / BN;
                nsl = 0;
                for (int e = tg.cb; e < tg.ce; ++e) nsl += (crec[e].ri + BK - 1) / BK;
                if (ntm <= 0 || ntn <= 0 || nsl == 0) continue;   // nothing to subtract
                tm = tn = 0;
                start_tile();
                active = true;
            }
            while (c < tg.ce) {
                if (k0 < cr.ri) {
                    const int m0 = tm * BM, n0 = tn * BN;
                    m.A = blk + cr.aoff + tg.row_lo + m0 + (int64_t)k0 * tg.nj;
                    m.lda = tg.nj;
                    m.B = WU + cr.boff + (int64_t)n0 * cr.ri + k0;
                    m.ldb = cr.ri;
                    m.kv = min(BK, cr.ri - k0);
                    m.mv = mv;
                    m.nv = nv;
                    m.n = nmma;
                    m.flags = (sl == 0 ? F_FIRST : 0) | (sl == nsl - 1 ? F_LAST : 0);
                    ++sl;
                    k0 += BK;
                    return true;
                }
                if (++c < tg.ce) cr = crec[c];
                k0 = 0;
            }
            if (++tn == ntn) { tn = 0; ++tm; }
            if (tm < ntm) start_tile();
            else active = false;
        }
    }
};

// registers of one slice: thread t holds 8 consecutive k of A row (t & 127) and of B
// column (t & 127), k half t >> 7
__device__ __forceinline__ void load_slice(const SliceMeta& m, int tid, float (&ra)[8], float (&rb)[8]) {
    const int line = tid & 127, h = tid >> 7;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = 8 * h + e;
        const bool kin = k < m.kv;
        ra[e] = (kin && line < m.mv) ? __ldg(m.A + line + (int64_t)k * m.lda) : 0.f;
        rb[e] = (kin && line < m.nv) ? __ldg(m.B + k + (int64_t)line * m.ldb) : 0.f;
    }
}

__device__ __forceinline__ void split4(const float* x, float4& hi, float4& lo) {
    hi.x = tc::to_tf32(x[0]); lo.x = tc::to_tf32(x[0] - hi.x);
    hi.y = tc::to_tf32(x[1]); lo.y = tc::to_tf32(x[1] - hi.y);
    hi.z = tc::to_tf32(x[2]); lo.z = tc::to_tf32(x[2] - hi.z);
    hi.w = tc::to_tf32(x[3]); lo.w = tc::to_tf32(x[3] - hi.w);
}

// hi / lo parts of the thread's 8 + 8 values into a stage (two 16-byte chunks each)
__device__ __forceinline__ void store_slice(unsigned char* st, int tid, const float (&ra)[8], const float (&rb)[8]) {
    const int line = tid & 127, h = tid >> 7;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int off = (line >> 3) * kSBO + (2 * h + g) * 128 + (line & 7) * 16;
        float4 hi, lo;
        split4(ra + 4 * g, hi, lo);
        *reinterpret_cast<float4*>(st + off) = hi;
        *reinterpret_cast<float4*>(st + kPart + off) = lo;
        split4(rb + 4 * g, hi, lo);
        *reinterpret_cast<float4*>(st + 2 * kPart + off) = hi;
        *reinterpret_cast<float4*>(st + 3 * kPart + off) = lo;
    }
}

// One stage of the ring from the producers: wait until the MMAs of its previous use
// are done, store, publish.  In drain mode (abort) nothing is waited for or stored.
__device__ __forceinline__ void put_stage(Ctrl* ctl, unsigned char* ring, int s, int tid, int flags, int n,
                                 const float (&ra)[8], const float (&rb)[8], long long budget) {
    const int st = s % kStages, use = s / kStages;
    const int lane = tid & 31;
    volatile int* ab = &ctl->abort;
    if (*ab) return;
    if (use >= 1 && lane == 0) wait_phase(&ctl->empty[st], (use - 1) & 1, ab, budget);
    __syncwarp();
    if (*ab) return;
    store_slice(ring + (size_t)st * kStageBytes, tid, ra, rb);
    if (tid == 0) ctl->hdr[st] = StageHdr{flags, n};
    tc::fence_proxy_async();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl->full[st]);
}

}  // namespace ws
}  // namespace h2rs
