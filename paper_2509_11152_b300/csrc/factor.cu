// Factorisation driver (Alg. 1): levels from the leaves up, colours in order, the
// batched kernels of Alg. 2 per colour, the level close, and the float64 dense LU of
// the top level.  One host synchronisation per level reads back the augmented ranks,
// which fix the sizes (and prefix-sum offsets) of the parent level.
#include <algorithm>
#include <chrono>
#include <functional>
#include <future>
#include <numeric>
#include <string>

#include "factor_impl.h"
#include "factor_kernels.cuh"

namespace h2rs {

// host stopwatch for h2_factor_stats.host_ms
struct HostTimer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double lap() {
        const auto t1 = std::chrono::steady_clock::now();
        const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        t0 = t1;
        return ms;
    }
};

enum { PH_AUG = 0, PH_PROJ = 1, PH_LU = 2, PH_SCHUR = 3, PH_CLOSE = 4, PH_TOP = 5, PH_LOAD = 6,
       PH_OTHER = 7 };


template <class T>
static LevelArgs<T> args_of(LevelRT& L, DevStatus* st) {
    LevelArgs<T> a{};
    a.level = L.l;
    a.cnt = L.cnt;
    a.n = L.d_n.as<int>();
    a.k = L.d_k.as<int>();
    a.kt = L.d_kt.as<int>();
    a.colour = L.d_colour.as<int>();
    a.blk_off = L.d_blk_off.as<int64_t>();
    a.brow = L.d_brow.as<int>();
    a.bcol = L.d_bcol.as<int>();
    a.blk = L.blk.as<T>();
    a.V_off = L.d_V_off.as<int64_t>();
    a.V = L.V.as<T>();
    a.Q_off = L.d_Q_off.as<int64_t>();
    a.Q = L.Q.as<T>();
    a.LU_off = L.d_LU_off.as<int64_t>();
    a.LU = L.LU.as<T>();
    a.DI = L.DI.as<T>();
    a.piv_off = L.d_piv_off.as<int64_t>();
    a.piv = L.piv.as<int>();
    a.WU_off = L.d_WU_off.as<int64_t>();
    a.WU = L.WU.as<T>();
    a.WL_off = L.d_WL_off.as<int64_t>();
    a.WL = L.WL.as<T>();
    a.WLld = L.d_WLld.as<int>();
    a.nb_ptr = L.d_nb_ptr.as<int>();
    a.nb_col = L.d_nb_col.as<int>();
    a.nbofs = L.d_nbofs.as<int>();
    a.Nsum = L.d_Nsum.as<int>();
    a.nb_blk = L.d_nb_blk.as<int>();
    a.nb_blkT = L.d_nb_blkT.as<int>();
    a.diag_blk = L.d_diag_blk.as<int>();
    a.eps_fill = L.d_eps.as<T>();
    a.force_kt = L.d_force.ptr ? L.d_force.as<int>() : nullptr;
    a.status = st;
    return a;
}

// Raise a kernel's dynamic shared memory limit to what the device allows beside the
// kernel's static shared memory; returns that limit.
template <class K>
static int raise_smem(K kern) {
    int dev = 0, optin = 0;
    H2_CUDA_CHECK(cudaGetDevice(&dev));
    H2_CUDA_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    H2_CUDA_CHECK(cudaFuncGetAttributes(&fa, kern));
    const int lim = optin - (int)fa.sharedSizeBytes;
    H2_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return lim;
}

template <class T, bool RIGHT>
static void launch_proj(int rpt, int nwork, int npan, int smem, cudaStream_t s, LevelArgs<T> ar, int c,
                        const int* box, const int* blk) {
    const dim3 g(nwork, npan);                        // y: 32-wide panel of the block
    if (rpt <= 1) k_proj<T, 1, RIGHT><<<g, 256, smem, s>>>(ar, c, box, blk);
    else if (rpt <= 2) k_proj<T, 2, RIGHT><<<g, 256, smem, s>>>(ar, c, box, blk);
    else if (rpt <= 4) k_proj<T, 4, RIGHT><<<g, 256, smem, s>>>(ar, c, box, blk);
    else if (rpt <= 8) k_proj<T, 8, RIGHT><<<g, 256, smem, s>>>(ar, c, box, blk);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the projection kernel"};
}

static int num_sms() {
    static const int n = [] {
        int dev = 0, v = 0;
        H2_CUDA_CHECK(cudaGetDevice(&dev));
        H2_CUDA_CHECK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        return v;
    }();
    return n;
}

// tensor-core projection (float32 factors only): one CTA per box of the colour
static void launch_proj_tc(bool, int, cudaStream_t, const LevelArgs<double>&, int, const int*, const int*,
                           const int*, long long) {}
static void launch_proj_tc(bool right, int nbx, cudaStream_t s, const LevelArgs<float>& ar, int c,
                           const int* boxes, const int* pj_ptr, const int* blks, long long budget) {
    static const bool ready = [] {
        H2_CUDA_CHECK(cudaFuncSetAttribute(k_proj_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, pj::kSmem));
        H2_CUDA_CHECK(cudaFuncSetAttribute(k_proj_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pj::kSmem));
        return true;
    }();
    (void)ready;
    if (right) k_proj_tc<true><<<nbx, pj::kThreads, pj::kSmem, s>>>(ar, c, boxes, pj_ptr, blks, budget);
    else k_proj_tc<false><<<nbx, pj::kThreads, pj::kSmem, s>>>(ar, c, boxes, pj_ptr, blks, budget);
}


static void launch_schur(bool, int ntile, cudaStream_t s, const LevelArgs<double>& ar, int c, int tg0,
                         const int* tb, const int* tp, const int* cb, const int* ca, const int* ck, const SchurTgt*,
                         const SchurCon*, const unsigned char*, const unsigned char*, long long) {
    k_schur<double><<<ntile, 256, 0, s>>>(ar, c, tg0, tb, tp, cb, ca, ck);
}

static void launch_schur(bool tensor, int ntile, cudaStream_t s, const LevelArgs<float>& ar, int c, int tg0,
                         const int* tb, const int* tp, const int* cb, const int* ca, const int* ck,
                         const SchurTgt* trec, const SchurCon* crec, const unsigned char* pA,
                         const unsigned char* pB, long long budget) {
    if (!tensor) {
        k_schur<float><<<ntile, 256, 0, s>>>(ar, c, tg0, tb, tp, cb, ca, ck);
        return;
    }
    // tensor path: ntile = number of targets of the colour, trec offset to the first;
    // persistent CTAs, two per SM
    static const int nsm = [] {
        H2_CUDA_CHECK(cudaFuncSetAttribute(k_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, ws::kSmem));
        int dev = 0, n = 0;
        H2_CUDA_CHECK(cudaGetDevice(&dev));
        H2_CUDA_CHECK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        return n;
    }();
    const int grid = std::min(ntile, ws::kCtasPerSm * nsm);
    k_schur_tc<<<grid, ws::kThreads, ws::kSmem, s>>>(ar, trec, crec, ntile, pA, pB, budget);
}

// operand packing of the tensor-core Schur update (float32 factors only)
static void launch_pack(int, int, cudaStream_t, const LevelArgs<double>&, const int*, const int*, const int64_t*,
                        unsigned char*, unsigned char*) {}
static void launch_pack(int npk, int c, cudaStream_t s, const LevelArgs<float>& ar, const int* box,
                        const int* pos, const int64_t* off, unsigned char* pA, unsigned char* pB) {
    k_schur_pack<<<dim3(npk, 2), 256, 0, s>>>(ar, c, box, pos, off, pA, pB);
}

// W_U (left) / W_L by triangular solves: CTAs per box enough for about four per SM
// (at most 8), the factors staged in shared memory when r_max^2 words fit
template <class T, bool LEFT, int RU>
static void launch_wtrsm_ru(int nmax, int nbmax, int nbx, cudaStream_t s, const LevelArgs<T>& ar,
                            const int* boxes) {
    static const int lim = std::min(raise_smem(k_wtrsm<T, LEFT, RU, true>), raise_smem(k_wtrsm<T, LEFT, RU, false>));
    const size_t sm = wtrsm_smem<T>(nmax * nmax, nbmax);
    const dim3 grid((unsigned)nbx, (unsigned)std::max(1, std::min(8, (4 * num_sms() + nbx - 1) / nbx)));
    if (sm <= (size_t)lim) {
        k_wtrsm<T, LEFT, RU, true><<<grid, 256, sm, s>>>(ar, boxes, nmax * nmax);
    } else {
        const size_t sm0 = wtrsm_smem<T>(0, nbmax);
        if (sm0 > (size_t)lim) throw Error{H2_ERR_ARG, "near field too large for the triangular solves"};
        k_wtrsm<T, LEFT, RU, false><<<grid, 256, sm0, s>>>(ar, boxes, 0);
    }
}

template <class T, bool LEFT>
static void launch_wtrsm(int nmax, int nbmax, int nbx, cudaStream_t s, const LevelArgs<T>& ar, const int* boxes) {
    if (nmax <= 32) launch_wtrsm_ru<T, LEFT, 1>(nmax, nbmax, nbx, s, ar, boxes);
    else if (nmax <= 64) launch_wtrsm_ru<T, LEFT, 2>(nmax, nbmax, nbx, s, ar, boxes);
    else if (nmax <= 128) launch_wtrsm_ru<T, LEFT, 4>(nmax, nbmax, nbx, s, ar, boxes);
    else if (nmax <= 256) launch_wtrsm_ru<T, LEFT, 8>(nmax, nbmax, nbx, s, ar, boxes);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the triangular solves"};
}

// D_RR^-1 from the LU factors, CTAs per box as for the triangular solves
template <class T, int RU>
static void launch_inverse_ru(int nmax, int nbx, cudaStream_t s, const LevelArgs<T>& ar, const int* boxes) {
    static const int lim = raise_smem(k_inverse<T, RU, true>);
    const size_t sm = (size_t)nmax * nmax * sizeof(T);
    const dim3 grid((unsigned)nbx, (unsigned)std::max(1, std::min(8, (4 * num_sms() + nbx - 1) / nbx)));
    if (sm <= (size_t)lim) k_inverse<T, RU, true><<<grid, 256, sm, s>>>(ar, boxes, nmax * nmax);
    else k_inverse<T, RU, false><<<grid, 256, 0, s>>>(ar, boxes, 0);
}

template <class T>
static void launch_inverse(int nmax, int nbx, cudaStream_t s, const LevelArgs<T>& ar, const int* boxes) {
    if (nmax <= 32) launch_inverse_ru<T, 1>(nmax, nbx, s, ar, boxes);
    else if (nmax <= 64) launch_inverse_ru<T, 2>(nmax, nbx, s, ar, boxes);
    else if (nmax <= 128) launch_inverse_ru<T, 4>(nmax, nbx, s, ar, boxes);
    else if (nmax <= 256) launch_inverse_ru<T, 8>(nmax, nbx, s, ar, boxes);
    else throw Error{H2_ERR_ARG, "box size above 256 is not supported by the inverse"};
}

template <class T>
struct SmemLimits {
    int basis, lu, proj_l, proj_r, gather;
};

template <class T>
static const SmemLimits<T>& smem_limits() {
    static SmemLimits<T> lim = [] {
        SmemLimits<T> x{};
        x.basis = std::min(raise_smem(k_basis<T, false>), raise_smem(k_basis<T, true>));
        x.lu = raise_smem(k_lu<T>);
        x.proj_l = std::min({raise_smem(k_proj<T, 1, false>), raise_smem(k_proj<T, 2, false>),
                             raise_smem(k_proj<T, 4, false>), raise_smem(k_proj<T, 8, false>)});
        x.proj_r = std::min({raise_smem(k_proj<T, 1, true>), raise_smem(k_proj<T, 2, true>),
                             raise_smem(k_proj<T, 4, true>), raise_smem(k_proj<T, 8, true>)});
        x.gather = std::min(raise_smem(k_aug_gather<T, true>), raise_smem(k_aug_gather<T, false>));

        return x;
    }();
    return lim;
}

// every launch is checked before anything that depends on it is enqueued
#define H2_LAUNCHED() H2_CUDA_CHECK(cudaGetLastError())

template <class T>
FactorImpl<T>::FactorImpl(const MatrixObj* A_, const h2_factor_opts& o) {
    (void)smem_limits<T>();
    A = A_;
    eps_lu = o.eps_lu;
    norm_a = o.norm_a;
    precision = o.precision;
    tensor_schur = o.precision == H2_PREC_TF32X3;
    w_inverse = tensor_schur;
    if (o.flags & H2_FLAG_W_TRIANGULAR) w_inverse = false;
    if (o.flags & H2_FLAG_W_INVERSE) w_inverse = true;
    H2_REQUIRE(!((o.flags & H2_FLAG_W_TRIANGULAR) && (o.flags & H2_FLAG_W_INVERSE)), H2_ERR_ARG,
               "H2_FLAG_W_TRIANGULAR and H2_FLAG_W_INVERSE exclude each other");
    norm_sys.assign(A->H.nsys, o.norm_a);
    if (o.sys_norm_a)
        for (int z = 0; z < A->H.nsys; ++z) {
            H2_REQUIRE(o.sys_norm_a[z] > 0 && std::isfinite(o.sys_norm_a[z]), H2_ERR_ARG,
                       "sys_norm_a entries must be > 0");
            norm_sys[z] = o.sys_norm_a[z];
        }
    time_kernels = (o.flags & H2_FLAG_TIME_KERNELS) != 0;
    if (o.force_ranks) {
        const Plan& P = A->plan;
        force_off.assign(P.levels.size() + 1, 0);
        for (size_t a = 0; a < P.levels.size(); ++a) force_off[a + 1] = force_off[a] + P.levels[a].cnt;
        force.assign(o.force_ranks, o.force_ranks + force_off.back());
        for (size_t a = 0; a < P.levels.size(); ++a)
            for (int i = 0; i < P.levels[a].cnt; ++i) {
                const int64_t g = P.levels[a].first + i;
                const int v = force[force_off[a] + i];
                H2_REQUIRE(v >= 0 && (a > 0 || v <= A->H.node_size[g]), H2_ERR_ARG,
                           "force_ranks: negative rank or rank above the box size");
            }
    }
    if (o.flags & H2_FLAG_DEBUG_SHORT_WAIT) wait_budget = 1;
    H2_REQUIRE(o.k_cap >= 0, H2_ERR_ARG, "k_cap must be >= 0");
    k_cap = o.k_cap;
    stream = static_cast<cudaStream_t>(o.stream);
    status.alloc(sizeof(DevStatus), stream);
}

template <class T>
FactorImpl<T>::~FactorImpl() {
    for (auto e : ev) cudaEventDestroy(e);
    for (auto e : kev) cudaEventDestroy(e);
}

template <class T>
void FactorImpl<T>::kbegin(int id) {
    count_launch();
    if (!time_kernels) return;
    cudaEvent_t e;
    H2_CUDA_CHECK(cudaEventCreate(&e));
    H2_CUDA_CHECK(cudaEventRecord(e, stream));
    kev.push_back(e);
    kev_id.push_back(id);
}

template <class T>
void FactorImpl<T>::kend() {
    if (!time_kernels) return;
    cudaEvent_t e;
    H2_CUDA_CHECK(cudaEventCreate(&e));
    H2_CUDA_CHECK(cudaEventRecord(e, stream));
    kev.push_back(e);
    kev_id.push_back(-1);
}

template <class T>
void FactorImpl<T>::mark(int phase) {
    cudaEvent_t e;
    H2_CUDA_CHECK(cudaEventCreate(&e));
    H2_CUDA_CHECK(cudaEventRecord(e, stream));
    ev.push_back(e);
    ev_phase.push_back(phase);
}

template <class T>
void FactorImpl<T>::check_status(const char* where) {
    DevStatus h{};
    H2_CUDA_CHECK(cudaMemcpyAsync(&h, status.ptr, sizeof(h), cudaMemcpyDeviceToHost, stream));
    H2_CUDA_CHECK(cudaStreamSynchronize(stream));
    H2_CUDA_CHECK(cudaGetLastError());
    if (h.code != 0) {
        stats.error_level = h.level;
        stats.error_box = h.box;
        throw Error{h.code, std::string(where) + ": device status " + std::to_string(h.code) +
                                " at level " + std::to_string(h.level) + " box " +
                                std::to_string(h.box)};
    }
}

template <class T>
static int64_t track(FactorImpl<T>* F, DevBuf& b, size_t bytes, cudaStream_t s) {
    b.alloc(bytes, s);
    F->bytes_now += (int64_t)bytes;
    F->stats.peak_bytes = std::max(F->stats.peak_bytes, F->bytes_now);
    return (int64_t)bytes;
}

template <class T>
static void untrack(FactorImpl<T>* F, DevBuf& b) {
    F->bytes_now -= (int64_t)b.bytes;
    b.release();
}

// ------------------------------------------------------------------ level setup
template <class T>
void FactorImpl<T>::setup_level(size_t a) {
    const Plan& P = A->plan;
    const HostStructure& H = A->H;
    const bool is_top = a == P.levels.size();
    const LevelStruct& S = is_top ? P.toplev : P.levels[a];
    LevelRT& L = lv[a];
    L.S = &S;
    L.l = S.l;
    L.cnt = S.cnt;
    L.n.assign(S.cnt, 0);
    L.k.assign(S.cnt, 0);
    for (int i = 0; i < S.cnt; ++i) {
        if (a == 0 && S.l == H.d) L.n[i] = (int)H.node_size[S.first + i];
        else L.n[i] = lv[a - 1].kt[2 * i] + lv[a - 1].kt[2 * i + 1];
        L.k[i] = (int)H.rank[S.first + i];
    }
    // boxes of dense top matrices: offsets inside their system's matrix
    L.ttoff.assign(S.cnt, 0);
    L.tsys.assign(S.cnt, 0);
    for (int i : S.top_boxes) {
        const int z = H.sys[S.first + i];
        L.tsys[i] = z;
        L.ttoff[i] = sys_nt[z];
        sys_nt[z] += L.n[i];
    }
    std::vector<T> eps(S.cnt);
    for (int i = 0; i < S.cnt; ++i) eps[i] = (T)(eps_lu * norm_sys[H.sys[S.first + i]]);
    const int nb = S.nblocks();
    L.brow.resize(nb);
    L.blk_off.assign(nb + 1, 0);
    for (int i = 0; i < S.cnt; ++i)
        for (int b = S.bptr[i]; b < S.bptr[i + 1]; ++b) {
            L.brow[b] = i;
            L.blk_off[b + 1] = L.blk_off[b] + (int64_t)L.n[i] * L.n[S.bcol[b]];
        }
    auto prefix = [&](std::vector<int64_t>& off, auto f) {
        off.assign(S.cnt + 1, 0);
        for (int i = 0; i < S.cnt; ++i) off[i + 1] = off[i] + f(i);
    };
    prefix(L.V_off, [&](int i) { return (int64_t)L.n[i] * L.k[i]; });
    prefix(L.voff, [&](int i) { return (int64_t)L.n[i]; });
    L.vtot = L.voff[S.cnt];
    cudaStream_t s = stream;
    upload(L.d_n, L.n, s);
    upload(L.d_k, L.k, s);
    L.d_colour.ptr = S.dev.colour.ptr;
    L.d_brow.ptr = S.dev.brow.ptr;
    L.d_bcol.ptr = S.dev.bcol.ptr;
    L.d_top_boxes.ptr = S.dev.top_boxes.ptr;
    L.d_skel_boxes.ptr = S.dev.skel_boxes.ptr;
    L.d_nb_ptr.ptr = S.dev.nb_ptr.ptr;
    L.d_nb_col.ptr = S.dev.nb_col.ptr;
    L.d_nb_blk.ptr = S.dev.nb_blk.ptr;
    L.d_nb_blkT.ptr = S.dev.nb_blkT.ptr;
    L.d_diag_blk.ptr = S.dev.diag_blk.ptr;
    L.d_fl_tbox.ptr = S.dev.fl_tbox.ptr;
    L.d_fl_tptr.ptr = S.dev.fl_tptr.ptr;
    L.d_fl_ci.ptr = S.dev.fl_ci.ptr;
    L.d_fl_cpos.ptr = S.dev.fl_cpos.ptr;
    upload(L.d_blk_off, L.blk_off, s);
    upload(L.d_V_off, L.V_off, s);
    upload(L.d_voff, L.voff, s);
    upload(L.d_ttoff, L.ttoff, s);
    upload(L.d_tsys, L.tsys, s);
    upload(L.d_eps, eps, s);
    if (!force.empty() && !is_top) {
        const std::vector<int> fk(force.begin() + force_off[a], force.begin() + force_off[a + 1]);
        upload(L.d_force, fk, s);
    }
    L.kt.assign(S.cnt, 0);
    upload(L.d_kt, L.kt, s);
    track(this, L.blk, std::max<int64_t>(1, L.blk_off[nb]) * sizeof(T), s);
    if (is_top) return;
    track(this, L.V, std::max<int64_t>(1, L.V_off[S.cnt]) * sizeof(T), s);
    // factor data only for the boxes skeletonised here
    auto sk = [&](int i) { return S.state[i] == 1; };
    prefix(L.Q_off, [&](int i) { return sk(i) ? (int64_t)L.n[i] * L.n[i] : 0; });
    L.LU_off = L.Q_off;
    prefix(L.piv_off, [&](int i) { return sk(i) ? (int64_t)L.n[i] : 0; });
    L.Nsum.assign(S.cnt, 0);
    L.nbofs.assign(S.nb_col.size(), 0);
    for (int i = 0; i < S.cnt; ++i) {
        int o = 0;
        for (int p = S.nb_ptr[i]; p < S.nb_ptr[i + 1]; ++p)
            if (S.nb_col[p] != i) { L.nbofs[p] = o; o += L.n[S.nb_col[p]]; }
        L.Nsum[i] = o;
        for (int p = S.nb_ptr[i]; p < S.nb_ptr[i + 1]; ++p)
            if (S.nb_col[p] == i) L.nbofs[p] = o;
    }
    L.WLld.resize(S.cnt);
    for (int i = 0; i < S.cnt; ++i) L.WLld[i] = L.Nsum[i] + L.n[i];
    prefix(L.WU_off, [&](int i) { return sk(i) ? (int64_t)L.n[i] * L.WLld[i] : 0; });
    L.WL_off = L.WU_off;
    upload(L.d_Q_off, L.Q_off, s);
    upload(L.d_LU_off, L.LU_off, s);
    upload(L.d_piv_off, L.piv_off, s);
    upload(L.d_WU_off, L.WU_off, s);
    upload(L.d_WL_off, L.WL_off, s);
    upload(L.d_WLld, L.WLld, s);
    upload(L.d_nbofs, L.nbofs, s);
    upload(L.d_Nsum, L.Nsum, s);
    track(this, L.Q, std::max<int64_t>(1, L.Q_off[S.cnt]) * sizeof(T), s);
    track(this, L.LU, std::max<int64_t>(1, L.LU_off[S.cnt]) * sizeof(T), s);
    track(this, L.DI, std::max<int64_t>(1, L.Q_off[S.cnt]) * sizeof(T), s);
    track(this, L.piv, std::max<int64_t>(1, L.piv_off[S.cnt]) * sizeof(int), s);
    track(this, L.WU, std::max<int64_t>(1, L.WU_off[S.cnt]) * sizeof(T), s);
    track(this, L.WL, std::max<int64_t>(1, L.WL_off[S.cnt]) * sizeof(T), s);
}

// size-dependent work data of one level (the structural lists live in the plan)
struct ColourWork {
    std::vector<int64_t> ybase, ylead, wbase;             // basis: per box
    std::vector<int64_t> scratch_need;                     // per colour (elements)
    std::vector<int> smem_basis, w_in_smem, smem_gather, gather_pc, gather_vs, nmax, nbmax;
    std::vector<int> wu_box, wu_mn, wu_cptr, wl_box, wl_mn, wl_cptr;   // W_U / W_L GEMM tiles (TF32X3)
};

// Algorithmic flops and bytes of one level's phases (the roofline definitions of the
// kernels' work units), from the plan and the level's sizes and ranks.
LevelCounts level_counts(const LevelStruct& S, const LevelRT& L, double w) {
    LevelCounts R{};
    auto account = [&](int ph, double f, double b) { R.flops[ph] += f; R.bytes[ph] += b; };
    const int nc = S.ncolour;
    for (int c = 0; c < nc; ++c) {
        for (int i : S.cboxes[c]) {
            const double n = L.n[i], kt = L.kt[i], r = n - kt;
            double live = 0;
            for (int b = S.bptr[i]; b < S.bptr[i + 1]; ++b)
                if (S.bkind[b] == 1 && S.first_touch[b] < c) {
                    const int j = S.bcol[b];
                    live += (S.colour[j] < c) ? L.kt[j] : L.n[j];
                }
            account(PH_AUG, 4.0 * n * L.k[i] * live + 2.0 * live * n * n + 4.0 * n * n * kt,
                    w * (live * n + n * n));
            double nsum = 0, pbytes = 0;
            for (int b = S.bptr[i]; b < S.bptr[i + 1]; ++b) {
                const bool lv_ = S.bkind[b] == 0 || S.first_touch[b] < c;
                if (!lv_) continue;
                const int jb = S.bcol[b];
                const double nj = S.colour[jb] < c ? L.kt[jb] : L.n[jb];   // rectangular fill
                pbytes += 4.0 * n * nj * w;
                account(PH_PROJ, 4.0 * n * n * nj, 0);
            }
            account(PH_PROJ, 0, pbytes + n * n * w);
            for (int p = S.nb_ptr[i]; p < S.nb_ptr[i + 1]; ++p)
                if (S.nb_col[p] != i) nsum += L.n[S.nb_col[p]];
            const double ncol = nsum + kt;
            account(PH_LU, 2.0 / 3.0 * r * r * r + 4.0 * r * r * ncol, w * (4.0 * r * ncol + r * r));
        }
        // Schur: targets read and written once; each contributor's operands D_{j,i_R}
        // and W_U^i read once per colour (rows / columns of boxes eliminated before or
        // in this colour: skeleton part only, rectangular fill)
        auto live_lines = [&](int j) -> double { return S.colour[j] <= c ? L.kt[j] : L.n[j]; };
        for (int t = S.sch_cptr[c]; t < S.sch_cptr[c + 1]; ++t) {
            const int tb = S.sch_tblk[t];
            const double m = live_lines(L.brow[tb]), nn = live_lines(S.bcol[tb]);
            double fl = 0, reread = 0;
            for (int e = S.sch_tptr[t]; e < S.sch_tptr[t + 1]; ++e) {
                const double r = L.n[S.sch_ci[e]] - L.kt[S.sch_ci[e]];
                fl += 2.0 * m * nn * r;
                reread += w * r * (m + nn);
            }
            account(PH_SCHUR, fl, 2.0 * m * nn * w);
            R.schur_reread += reread;
        }
        for (int i : S.cboxes[c]) {
            const double r = L.n[i] - L.kt[i];
            double lines = 0;
            for (int p = S.nb_ptr[i]; p < S.nb_ptr[i + 1]; ++p) lines += live_lines(S.nb_col[p]);
            account(PH_SCHUR, 0, 2.0 * w * r * lines);
        }
    }
    return R;
}

template <class T>
void FactorImpl<T>::run_level(size_t a) {
    LevelRT& L = lv[a];
    const LevelStruct& S = *L.S;
    const MatrixObj& M = *A;
    cudaStream_t s = stream;
    LevelArgs<T> ar = args_of<T>(L, status.as<DevStatus>());
    if (a == 0) {
        kbegin(H2_K_LOAD);
        k_leaf_load<T><<<S.nblocks(), 256, 0, s>>>(ar, M.D.as<double>(), M.d_D_off.as<int64_t>(),
                                                 S.dev.near_entry.as<int64_t>());
        kend();
        H2_LAUNCHED();
        std::vector<int64_t> uoff(M.H.U_off.begin(), M.H.U_off.end());
        DevBuf d_uoff;
        upload(d_uoff, uoff, s);
        kbegin(H2_K_LOAD);
        k_leaf_basis<T><<<S.cnt, 256, 0, s>>>(ar, L.V.as<T>(), M.U.as<double>(), d_uoff.as<int64_t>());
        kend();
        H2_LAUNCHED();
        H2_CUDA_CHECK(cudaGetLastError());
        mark(PH_LOAD);
        double bytes = 0;
        for (int b = 0; b < S.nblocks(); ++b)
            bytes += (double)(L.blk_off[b + 1] - L.blk_off[b]) * (S.bkind[b] == 0 ? 8 + sizeof(T) : sizeof(T));
        account(PH_LOAD, 0, bytes);
    }
    // ---------------- size-dependent work data (the structural lists live in the plan)
    HostTimer ht;
    ColourWork W;
    const int nc = S.ncolour;
    const int PW = 32;
    const int nbox_all = S.cbox_ptr[nc];
    W.ybase.resize(nbox_all);
    W.ylead.resize(nbox_all);
    W.wbase.resize(nbox_all);
    W.wu_cptr.push_back(0);
    W.wl_cptr.push_back(0);
    int nmax_level = 1;
    for (int v : L.n) nmax_level = std::max(nmax_level, v);
    for (int c = 0; c < nc; ++c) {
        int64_t ysum = 0, wsum = 0;
        int nmax = 0, kmax = 0, csz = 0;
        for (int q = S.cbox_ptr[c]; q < S.cbox_ptr[c + 1]; ++q) {
            const int i = S.cboxes[c][q - S.cbox_ptr[c]];
            const int n = L.n[i];
            nmax = std::max(nmax, n);
            int64_t yrows = 0;
            for (int g = S.seg_ptr[q]; g < S.seg_ptr[q + 1]; ++g) yrows += L.n[S.seg_j[g]];
            W.ybase[q] = ysum;
            W.ylead[q] = yrows;
            ysum += yrows * n;
            W.wbase[q] = wsum;
            wsum += (int64_t)n * (n + 1);
            kmax = std::max(kmax, L.k[i]);
            csz = std::max(csz, basis_chunk_elems(n));
            const int wide = L.Nsum[i] + n;          // bound of the width sum n_j + k~_i
            if (w_inverse)                           // GEMM tiles (the triangular solves take a CTA per box)
                for (int tm = 0; tm * 64 < n; ++tm)
                    for (int tn = 0; tn * 64 < wide; ++tn) {
                        W.wu_box.push_back(i);
                        W.wu_mn.push_back((tm << 16) | tn);
                        W.wl_box.push_back(i);
                        W.wl_mn.push_back((tn << 16) | tm);
                    }
        }
        for (int q = S.cbox_ptr[c]; q < S.cbox_ptr[c + 1]; ++q) W.wbase[q] += ysum;   // after the Y^T rows
        W.wu_cptr.push_back((int)W.wu_box.size());
        W.wl_cptr.push_back((int)W.wl_box.size());
        const size_t base = (size_t)(csz + 2 * nmax + 33) * sizeof(T) + 16;
        const size_t wsm = (size_t)nmax * (nmax + 1) * sizeof(T);
        const auto& lim = smem_limits<T>();
        // gather: the widest chunk of F that fits, with V staged when it fits too
        size_t gsm = 0;
        int gpc = 0, gvs = 0;
        for (int vs = 1; vs >= 0 && !gpc; --vs)
            for (int pc : {64, 32, 16}) {
                const size_t need = ((size_t)(nmax + 1) * pc + (size_t)(kmax + 1) * pc +
                                     (vs ? (size_t)(nmax + 1) * kmax : 0)) * sizeof(T);
                if (need <= (size_t)lim.gather) { gsm = need; gpc = pc; gvs = vs; break; }
            }
        H2_REQUIRE(gpc > 0 && base <= (size_t)lim.basis &&
                       (size_t)2 * 32 * ((nmax + 31) / 32 * 32 + 1) * sizeof(T) <= (size_t)std::min(lim.proj_l, lim.proj_r) &&
                       nmax <= 256,
                   H2_ERR_ARG, "box size too large for the shared-memory kernels");
        W.gather_pc.push_back(gpc);
        W.gather_vs.push_back(gvs);
        const int in_sm = base + wsm <= (size_t)lim.basis;
        W.w_in_smem.push_back(in_sm);
        W.smem_basis.push_back((int)(base + (in_sm ? wsm : 0)));
        W.smem_gather.push_back((int)gsm);
        W.nmax.push_back(nmax);
        int nbm = 1;
        for (int q = S.cbox_ptr[c]; q < S.cbox_ptr[c + 1]; ++q) {
            const int i = S.cboxes[c][q - S.cbox_ptr[c]];
            nbm = std::max(nbm, S.nb_ptr[i + 1] - S.nb_ptr[i]);
        }
        W.nbmax.push_back(nbm);
        W.scratch_need.push_back(ysum + (in_sm ? 0 : wsum));
    }
    stats.host_ms[0] += ht.lap();
    int64_t scratch_max = 1;
    for (auto v : W.scratch_need) scratch_max = std::max(scratch_max, v);
    DevBuf scratch;
    track(this, scratch, scratch_max * sizeof(T), s);
    DevBuf d_ybase, d_ylead, d_wbase, d_wu_box, d_wu_mn, d_wl_box, d_wl_mn, d_ynorm2;
    d_ynorm2.alloc(std::max(1, nbox_all) * sizeof(double), s);
    H2_CUDA_CHECK(cudaMemsetAsync(d_ynorm2.ptr, 0, std::max(1, nbox_all) * sizeof(double), s));
    upload(d_ybase, W.ybase, s);
    upload(d_ylead, W.ylead, s);
    upload(d_wbase, W.wbase, s);
    upload(d_wu_box, W.wu_box, s);
    upload(d_wu_mn, W.wu_mn, s);
    upload(d_wl_box, W.wl_box, s);
    upload(d_wl_mn, W.wl_mn, s);
    const DevBuf &d_tgt_blk = S.dev.sch_tblk, &d_tgt_ptr = S.dev.sch_tptr, &d_c_box = S.dev.sch_ci,
                 &d_c_ablk = S.dev.sch_cA, &d_c_kpos = S.dev.sch_ckpos;
    DevBuf d_trec, d_crec;                                 // Schur records (tensor-core path)
    // packed operands of the tensor-core Schur update: one region per near-field
    // position of every box, offsets restarting in every colour and bounded by the box
    // sizes (the ranks are not known here); the buffers fit the largest colour
    DevBuf d_pk_off, packA, packB;
    if (tensor_schur) {
        std::vector<int64_t> pk(S.nb_col.size() + 1, 0);
        int64_t mx = 256;
        for (int c = 0; c < nc; ++c) {
            int64_t off = 0;
            for (int q = S.pk_cptr[c]; q < S.pk_cptr[c + 1]; ++q) {
                const int p = S.pk_pos[q];
                pk[p] = off;
                off += ws::pack_region_bytes(L.n[S.pk_box[q]], L.n[S.nb_col[p]]);
            }
            mx = std::max(mx, off);
        }
        upload(d_pk_off, pk, s);
        track(this, packA, mx, s);
        track(this, packB, mx, s);
    }
    if (tensor_schur) {
        d_trec.alloc(std::max<size_t>(1, S.sch_tblk.size()) * sizeof(SchurTgt), s);
        d_crec.alloc(std::max<size_t>(1, S.sch_ci.size()) * sizeof(SchurCon), s);
    }
    stats.host_ms[1] += ht.lap();
    for (int c = 0; c < nc; ++c) {
        const int b0 = S.cbox_ptr[c], nbx = S.cbox_ptr[c + 1] - b0;
        if (nbx == 0) continue;
        ColourLists CL{};
        CL.boxes = S.dev.cboxes.as<int>() + b0;
        CL.seg_ptr = S.dev.seg_ptr.as<int>() + b0;  // per-box pointers into global seg arrays
        CL.seg_blk = S.dev.seg_blk.as<int>();
        CL.seg_j = S.dev.seg_j.as<int>();
        CL.ybase = d_ybase.as<int64_t>() + b0;
        CL.ylead = d_ylead.as<int64_t>() + b0;
        CL.wbase = d_wbase.as<int64_t>() + b0;
        CL.ynorm2 = d_ynorm2.as<double>() + b0;
        const int s0 = S.seg_cptr[c], ns = S.seg_cptr[c + 1] - s0;
        // ---- augmentation
        if (ns > 0) {
            ColourLists CG = CL;
            CG.seg_blk = S.dev.seg_blk.as<int>() + s0;
            CG.seg_j = S.dev.seg_j.as<int>() + s0;
            kbegin(H2_K_GATHER);
            if (W.gather_vs[c])
                k_aug_gather<T, true><<<ns, 256, W.smem_gather[c], s>>>(ar, CG, c, S.dev.seg_slot.as<int>() + s0, s0,
                                                                        W.gather_pc[c], scratch.as<T>());
            else
                k_aug_gather<T, false><<<ns, 256, W.smem_gather[c], s>>>(ar, CG, c, S.dev.seg_slot.as<int>() + s0,
                                                                         s0, W.gather_pc[c], scratch.as<T>());
            kend();
            H2_LAUNCHED();
        }
        kbegin(H2_K_BASIS);
        if (W.nmax[c] <= 128)
            k_basis<T, false><<<nbx, 256, W.smem_basis[c], s>>>(ar, CL, c, scratch.as<T>(), scratch.as<T>(),
                                                                W.w_in_smem[c]);
        else
            k_basis<T, true><<<nbx, 256, W.smem_basis[c], s>>>(ar, CL, c, scratch.as<T>(), scratch.as<T>(),
                                                               W.w_in_smem[c]);
        kend();
        H2_LAUNCHED();
        H2_CUDA_CHECK(cudaGetLastError());
        mark(PH_AUG);
        // ---- projection + fill truncation
        const int pj0 = S.pj_cptr[c], npj = S.pj_cptr[c + 1] - pj0;
        const int smp = 2 * PW * ((W.nmax[c] + 31) / 32 * 32 + 1) * (int)sizeof(T);
        const int rpt = (W.nmax[c] + 31) / 32;
        const int npan = (nmax_level + PW - 1) / PW;        // panels of the other dimension
        // tensor cores for the float32 factor with split-TF32 products on colours with at
        // least one box per SM whose boxes all have 65..128 points (one CTA per box: it
        // pays where every SM has a box of full-width tiles), the FMA pipes otherwise
        const bool proj_tc = tensor_schur && W.nmax[c] <= pj::BM && W.nmax[c] > pj::BM / 2 && nbx >= num_sms();
        for (int side = 0; side < 2 && npj; ++side) {
            kbegin(H2_K_PROJ);
            if (proj_tc)
                launch_proj_tc(side == 1, nbx, s, ar, c, S.dev.cboxes.as<int>() + b0, S.dev.pj_ptr.as<int>() + b0,
                               side == 0 ? S.dev.pj_blk.as<int>() : S.dev.pj_blkT.as<int>(), wait_budget);
            else if (side == 0)
                launch_proj<T, false>(rpt, npj, npan, smp, s, ar, c, S.dev.pj_box.as<int>() + pj0,
                                      S.dev.pj_blk.as<int>() + pj0);
            else
                launch_proj<T, true>(rpt, npj, npan, smp, s, ar, c, S.dev.pj_box.as<int>() + pj0,
                                     S.dev.pj_blkT.as<int>() + pj0);
            kend();
            H2_LAUNCHED();
        }
        const int zf0 = S.zf_cptr[c], nzf = S.zf_cptr[c + 1] - zf0;
        if (nzf) {
            kbegin(H2_K_ZERO);
            k_zero_redundant<T><<<nzf, 256, 0, s>>>(ar, S.dev.zf_box.as<int>() + zf0, S.dev.zf_blk.as<int>() + zf0,
                                                    S.dev.zf_col.as<int>() + zf0);
            kend();
        }
        H2_LAUNCHED();
        H2_CUDA_CHECK(cudaGetLastError());
        mark(PH_PROJ);
        // ---- partial LU + triangular solves
        const size_t lu_sm = (size_t)W.nmax[c] * W.nmax[c] * sizeof(T);
        const int lu_in = lu_sm <= (size_t)smem_limits<T>().lu;
        kbegin(H2_K_LU);
        k_lu<T><<<nbx, 256, lu_in ? lu_sm : 0, s>>>(ar, S.dev.cboxes.as<int>() + b0, lu_in, w_inverse ? 0 : 1);
        kend();
        if (w_inverse) {                           // D_RR^-1 (counted with the LU)
            H2_LAUNCHED();
            kbegin(H2_K_LU);
            launch_inverse<T>(W.nmax[c], nbx, s, ar, S.dev.cboxes.as<int>() + b0);
            kend();
        }
        H2_LAUNCHED();
        const int wu0 = W.wu_cptr[c], nwu = W.wu_cptr[c + 1] - wu0;
        if (!w_inverse) {
            kbegin(H2_K_TRSM);
            launch_wtrsm<T, true>(W.nmax[c], W.nbmax[c], nbx, s, ar, S.dev.cboxes.as<int>() + b0);
            kend();
            H2_LAUNCHED();
            kbegin(H2_K_TRSM);
            launch_wtrsm<T, false>(W.nmax[c], W.nbmax[c], nbx, s, ar, S.dev.cboxes.as<int>() + b0);
            kend();
        } else if (nwu) {
            kbegin(H2_K_TRSM);
            k_wgemm<T, true><<<nwu, 256, 0, s>>>(ar, d_wu_box.as<int>() + wu0, d_wu_mn.as<int>() + wu0);
            kend();
        }
        H2_LAUNCHED();
        const int wl0 = W.wl_cptr[c], nwl = W.wl_cptr[c + 1] - wl0;
        if (nwl) {
            kbegin(H2_K_TRSM);
            k_wgemm<T, false><<<nwl, 256, 0, s>>>(ar, d_wl_box.as<int>() + wl0, d_wl_mn.as<int>() + wl0);
            kend();
        }
        H2_LAUNCHED();
        H2_CUDA_CHECK(cudaGetLastError());
        mark(PH_LU);
        if (tensor_schur) {
            const int q0 = S.pk_cptr[c], nq = S.pk_cptr[c + 1] - q0;
            if (nq) {
                kbegin(H2_K_PACK);
                launch_pack(nq, c, s, ar, S.dev.pk_box.as<int>() + q0, S.dev.pk_pos.as<int>() + q0,
                            d_pk_off.as<int64_t>(), packA.as<unsigned char>(), packB.as<unsigned char>());
                kend();
                H2_LAUNCHED();
            }
        }
        // ---- Schur update and zeroing of the eliminated rows / columns
        const int tg0 = S.sch_cptr[c], ntg = S.sch_cptr[c + 1] - tg0;
        const int ntile = ntg;                                             // one record / CTA per target
        if (ntile) {
            kbegin(H2_K_SCHUR);
            if (tensor_schur) {
                const int e0 = S.sch_tptr[tg0], ne = S.sch_tptr[tg0 + ntg] - e0;
                k_schur_prep<T><<<(unsigned)((ntg + ne + 255) / 256), 256, 0, s>>>(
                    ar, c, tg0, ntg, e0, ne, d_tgt_blk.as<int>(), d_tgt_ptr.as<int>(), d_c_box.as<int>(),
                    S.dev.sch_cjpos.as<int>(), d_c_kpos.as<int>(), d_pk_off.as<int64_t>(), d_trec.as<SchurTgt>(),
                    d_crec.as<SchurCon>());
                H2_LAUNCHED();
                count_launch();
            }
            launch_schur(tensor_schur, ntile, s, ar, c, tg0, d_tgt_blk.as<int>(), d_tgt_ptr.as<int>(),
                         d_c_box.as<int>(), d_c_ablk.as<int>(), d_c_kpos.as<int>(), d_trec.as<SchurTgt>() + tg0,
                         d_crec.as<SchurCon>(),
                         packA.as<unsigned char>(), packB.as<unsigned char>(), wait_budget);
            kend();
        }
        const int zn0 = S.zn_cptr[c], nzn = S.zn_cptr[c + 1] - zn0;
        if (nzn) {
            kbegin(H2_K_ZERO);
            k_zero_redundant<T><<<nzn, 256, 0, s>>>(ar, S.dev.zn_box.as<int>() + zn0, S.dev.zn_blk.as<int>() + zn0,
                                                    S.dev.zn_col.as<int>() + zn0);
            kend();
        }
        H2_LAUNCHED();
        H2_CUDA_CHECK(cudaGetLastError());
        mark(PH_SCHUR);
    }
    // ---------------- ranks back to the host (sizes of the parent level)
    ht.lap();
    check_status("factorize level");
    H2_CUDA_CHECK(cudaMemcpyAsync(L.kt.data(), L.d_kt.ptr, L.cnt * sizeof(int), cudaMemcpyDeviceToHost, s));
    H2_CUDA_CHECK(cudaStreamSynchronize(s));
    stats.host_ms[3] += ht.lap();
    if (k_cap > 0)
        for (int i = 0; i < L.cnt; ++i)
            if (L.kt[i] > k_cap) {
                throw Error{H2_ERR_RANK_CAP, "augmented rank " + std::to_string(L.kt[i]) + " of box " +
                                                 std::to_string(i) + " at level " + std::to_string(a) +
                                                 " exceeds k_cap " + std::to_string(k_cap)};
            }
    untrack(this, scratch);
    if (tensor_schur) {
        untrack(this, packA);
        untrack(this, packB);
    }
    // ---------------- algorithmic counts of this level (for roofline fractions): a host
    // loop over every box and Schur target, run on a worker thread so that the GPU goes
    // on with the next level meanwhile (summed at the end of the factorisation)
    counts.push_back(std::async(std::launch::async, level_counts, std::cref(S), std::cref(L), (double)sizeof(T)));
}

// ------------------------------------------------------------------ level close
template <class T>
void FactorImpl<T>::close_level(size_t a) {
    LevelRT& L = lv[a];
    LevelRT& Pn = lv[a + 1];
    const LevelStruct& S = *L.S;
    const MatrixObj& M = *A;
    cudaStream_t s = stream;
    LevelArgs<T> ar = args_of<T>(L, status.as<DevStatus>());
    const DevBuf &d_cd = S.dev.cl_dblk, &d_cf = S.dev.cl_fblk, &d_ca = S.dev.cl_adm;
    const int nbp = Pn.S->nblocks();
    if (nbp) {
        kbegin(H2_K_CLOSE);
        k_close_blocks<T><<<nbp, 256, 0, s>>>(ar, Pn.blk.as<T>(), Pn.d_blk_off.as<int64_t>(),
                                              Pn.d_brow.as<int>(), Pn.d_bcol.as<int>(), d_cd.as<int>(),
                                              d_cf.as<int>(), d_ca.as<int64_t>(), M.S.as<double>(),
                                              M.d_S_off.as<int64_t>());
        kend();
    }
    H2_LAUNCHED();
    if (a + 1 < lv.size() - 1) {          // the top level keeps no basis
        kbegin(H2_K_CLOSE);
        k_close_basis<T><<<Pn.cnt, 256, 0, s>>>(ar, Pn.V.as<T>(), Pn.d_V_off.as<int64_t>(),
                                                Pn.d_k.as<int>(), M.E.as<double>(),
                                                M.d_E_off.as<int64_t>(), L.S->first);
        kend();
    }
    H2_LAUNCHED();
    H2_CUDA_CHECK(cudaGetLastError());
    mark(PH_CLOSE);
    account(PH_CLOSE, 0, 2.0 * sizeof(T) * (double)Pn.blk_off.back());
    untrack(this, L.blk);
    untrack(this, L.V);
}

// ------------------------------------------------------------------ top level
// Dense float64 top matrices of the systems whose skeletonisation ends below level a:
// allocated here (their orders are now known) and assembled from the level's blocks,
// before the level close releases them.
template <class T>
void FactorImpl<T>::assemble_tops(size_t a) {
    LevelRT& L = lv[a];
    const LevelStruct& S = *L.S;
    if (S.top_boxes.empty()) return;
    const MatrixObj& M = *A;
    const Plan& P = M.plan;
    cudaStream_t s = stream;
    for (int z = 0; z < M.H.nsys; ++z) {
        if (P.sys_toplev[z] != S.l) continue;
        const int64_t n2 = sys_nt[z] * sys_nt[z];
        track(this, sys_Dt[z], std::max<int64_t>(1, n2) * sizeof(double), s);
        track(this, sys_piv[z], std::max<int64_t>(1, sys_nt[z]) * sizeof(int), s);
        H2_CUDA_CHECK(cudaMemsetAsync(sys_Dt[z].ptr, 0, std::max<int64_t>(1, n2) * sizeof(double), s));
        tops[z] = TopSys{sys_Dt[z].as<double>(), sys_piv[z].as<int>(), sys_nt[z]};
    }
    upload(d_tops, tops, s);
    std::vector<int> blist;
    for (int i : S.top_boxes)
        for (int b = S.bptr[i]; b < S.bptr[i + 1]; ++b) blist.push_back(b);
    if (blist.empty()) return;
    DevBuf d_blist;
    upload(d_blist, blist, s);
    const bool leaf = S.l == M.H.d;                  // float64 blocks straight from A
    const DevBuf& d_near = S.dev.near_entry;
    kbegin(H2_K_TOP);
    k_top_assemble<T><<<(unsigned)blist.size(), 256, 0, s>>>(
        d_blist.as<int>(), L.blk.as<T>(), L.d_blk_off.as<int64_t>(), leaf ? M.D.as<double>() : nullptr,
        M.d_D_off.as<int64_t>(), leaf ? d_near.as<int64_t>() : nullptr, L.d_brow.as<int>(), L.d_bcol.as<int>(),
        L.d_n.as<int>(), L.d_ttoff.as<int64_t>(), L.d_tsys.as<int>(), d_tops.as<TopSys>());
    kend();
    H2_LAUNCHED();
}

// Blocked LU with partial pivoting of every system's top matrix: one launch per
// kernel and panel for the whole batch.
template <class T>
void FactorImpl<T>::top_factor() {
    cudaStream_t s = stream;
    LevelRT& Tl = lv.back();
    assemble_tops(lv.size() - 1);
    const int nsys = (int)tops.size();
    nt = 0;
    int64_t ntmax = 0;
    sys_xt.assign(nsys + 1, 0);
    double flops = 0;
    for (int z = 0; z < nsys; ++z) {
        nt += sys_nt[z];
        ntmax = std::max(ntmax, sys_nt[z]);
        sys_xt[z + 1] = sys_xt[z] + sys_nt[z];
        flops += 2.0 / 3.0 * (double)sys_nt[z] * sys_nt[z] * sys_nt[z];
    }
    upload(d_tops, tops, s);
    upload(d_sys_nt, sys_nt, s);
    upload(d_sys_xt, sys_xt, s);
    const int NB = 64;
    for (int64_t j0 = 0; j0 < ntmax; j0 += NB) {
        const int jb = (int)std::min<int64_t>(NB, ntmax - j0);
        kbegin(H2_K_TOP);
        k_top_panel<<<nsys, 1024, 0, s>>>(d_tops.as<TopSys>(), j0, NB, status.as<DevStatus>());
        kend();
        H2_LAUNCHED();
        kbegin(H2_K_TOP);
        k_top_swap<<<dim3((unsigned)((ntmax + 255) / 256), nsys), 256, 0, s>>>(d_tops.as<TopSys>(), j0, NB);
        kend();
        H2_LAUNCHED();
        const int64_t rest = ntmax - j0 - jb;
        if (rest > 0) {
            kbegin(H2_K_TOP);
            k_top_trsm<<<dim3((unsigned)((rest + 127) / 128), nsys), 128, 0, s>>>(d_tops.as<TopSys>(), j0, NB);
            kend();
            H2_LAUNCHED();
            const unsigned g = (unsigned)((rest + 63) / 64);
            kbegin(H2_K_TOP);
            k_top_gemm<<<dim3(g, g, nsys), 256, 0, s>>>(d_tops.as<TopSys>(), j0, NB);
            kend();
            H2_LAUNCHED();
        }
    }
    H2_CUDA_CHECK(cudaGetLastError());
    untrack(this, Tl.blk);
    mark(PH_TOP);
    double tb = 0;
    for (int z = 0; z < nsys; ++z) tb += 16.0 * (double)sys_nt[z] * sys_nt[z];
    account(PH_TOP, flops, tb);
    check_status("top-level LU");
}

template <class T>
void FactorImpl<T>::factorize() {
    const Plan& P = A->plan;
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    ev_phase.clear();
    for (int p = 0; p < 8; ++p) stats.phase_ms[p] = stats.phase_flops[p] = stats.phase_bytes[p] = 0;
    stats.schur_reread_bytes = 0;
    counts.clear();
    stats.error_level = stats.error_box = -1;
    H2_CUDA_CHECK(cudaMemsetAsync(status.ptr, 0, sizeof(DevStatus), stream));
    lv.clear();
    lv.resize(P.levels.size() + 1);
    const int nsys = A->H.nsys;
    sys_nt.assign(nsys, 0);
    sys_Dt.clear();
    sys_Dt.resize(nsys);
    sys_piv.clear();
    sys_piv.resize(nsys);
    tops.assign(nsys, TopSys{nullptr, nullptr, 0});
    bytes_now = 0;
    stats.peak_bytes = 0;
    mark(-1);
    setup_level(0);
    for (int q = 0; q < 4; ++q) stats.host_ms[q] = 0;
    for (size_t a = 0; a < P.levels.size(); ++a) {
        run_level(a);
        HostTimer hs;
        assemble_tops(a);
        setup_level(a + 1);
        close_level(a);
        stats.host_ms[2] += hs.lap();
    }
    top_factor();
    H2_CUDA_CHECK(cudaStreamSynchronize(stream));
    for (auto& f : counts) {
        const LevelCounts R = f.get();
        for (int p = 0; p < 8; ++p) account(p, R.flops[p], R.bytes[p]);
        stats.schur_reread_bytes += R.schur_reread;
    }
    counts.clear();
    float total = 0;
    for (size_t e = 1; e < ev.size(); ++e) {
        float ms = 0;
        H2_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[e - 1], ev[e]));
        const int ph = ev_phase[e] >= 0 ? ev_phase[e] : PH_OTHER;
        stats.phase_ms[ph] += ms;
        total += ms;
    }
    stats.factor_ms = total;
    for (int q = 0; q < 16; ++q) { stats.kernel_ms[q] = 0; stats.kernel_launches[q] = 0; }
    for (size_t e = 0; e + 1 < kev.size(); ++e)
        if (kev_id[e] >= 0 && kev_id[e + 1] < 0) {
            float ms = 0;
            H2_CUDA_CHECK(cudaEventElapsedTime(&ms, kev[e], kev[e + 1]));
            stats.kernel_ms[kev_id[e]] += ms;
            stats.kernel_launches[kev_id[e]] += 1;
        }
    for (auto e : kev) cudaEventDestroy(e);
    kev.clear();
    kev_id.clear();
    stats.nlevels = (int)P.levels.size();
    stats.top_level = P.top;
    stats.top_size = nt;
    int64_t fb = 0;
    for (auto& L : lv) fb += L.Q.bytes + L.LU.bytes + L.DI.bytes + L.piv.bytes + L.WU.bytes + L.WL.bytes;
    for (int z = 0; z < nsys; ++z) fb += sys_Dt[z].bytes + sys_piv[z].bytes;
    stats.factor_bytes = fb;
    // layout export (levels 0 .. nlevels-1)
    lay_sizes.clear(); lay_ranks.clear(); lay_rowptr.clear(); lay_col.clear(); lay_offset.clear();
    lay_colour.clear(); lay_kind.clear();
    for (size_t a = 0; a < P.levels.size(); ++a) {
        const LevelRT& L = lv[a];
        const LevelStruct& S = *L.S;
        lay_sizes.emplace_back(L.n.begin(), L.n.end());
        lay_ranks.emplace_back(L.kt.begin(), L.kt.end());
        lay_rowptr.emplace_back(S.bptr.begin(), S.bptr.end());
        lay_col.emplace_back(S.bcol.begin(), S.bcol.end());
        lay_offset.emplace_back(L.blk_off.begin(), L.blk_off.end());
        lay_colour.emplace_back(S.colour.begin(), S.colour.end());
        lay_kind.emplace_back(S.bkind.begin(), S.bkind.end());
    }
}

std::unique_ptr<FactorBase> make_factor(const MatrixObj* A, const h2_factor_opts& o) {
    if (o.precision == H2_PREC_FP32 || o.precision == H2_PREC_TF32X3)
        return std::make_unique<FactorImpl<float>>(A, o);
    return std::make_unique<FactorImpl<double>>(A, o);
}

template struct FactorImpl<double>;
template struct FactorImpl<float>;

}  // namespace h2rs
