// Host-side factor object: per-level device buffers and the drivers of the
// factorisation (factor.cu) and of the solve / refinement (solve.cu).
#pragma once

#include <future>
#include <memory>

#include "factor_args.cuh"

namespace h2rs {

// Per-level state kept by the factor (the solve needs most of it).
struct LevelRT {
    int l = 0, cnt = 0;
    const LevelStruct* S = nullptr;
    std::vector<int> n, k, kt;
    std::vector<int64_t> blk_off, V_off, Q_off, LU_off, piv_off, WU_off, WL_off, voff;
    std::vector<int> WLld, Nsum, nbofs, brow;
    int64_t vtot = 0;
    // boxes of dense top matrices at this level: offset inside their system's matrix
    std::vector<int64_t> ttoff;
    std::vector<int> tsys;
    DevBuf d_ttoff, d_tsys, d_eps, d_force;
    // device: sizes and offsets of this factorisation
    DevBuf d_n, d_k, d_kt, d_blk_off;
    DevBuf d_V_off, d_Q_off, d_LU_off, d_piv_off, d_WU_off, d_WL_off, d_WLld;
    DevBuf d_nbofs, d_Nsum, d_voff;
    // device: the level's structure (views of the matrix's LevelStruct::dev)
    DevView d_colour, d_brow, d_bcol, d_top_boxes, d_skel_boxes, d_nb_ptr, d_nb_col, d_nb_blk, d_nb_blkT,
        d_diag_blk, d_fl_tbox, d_fl_tptr, d_fl_ci, d_fl_cpos;
    // device: factor data
    DevBuf Q, LU, DI, piv, WU, WL;
    // device: working data (freed after the level close)
    DevBuf blk, V;
};

// algorithmic flops / bytes of one level's phases (h2_factor_stats)
struct LevelCounts {
    double flops[8], bytes[8], schur_reread;
};
LevelCounts level_counts(const LevelStruct& S, const LevelRT& L, double w);

struct FactorBase {
    virtual ~FactorBase() = default;
    virtual void factorize() = 0;
    // x <- A^-1 b in place; b is float64, device, n x nrhs with leading dimension ldb
    // x = M^-1 b in place; wide: float64 vectors and arithmetic whatever the factor's
    // storage precision (a fixed linear operator for Krylov refinement)
    virtual void solve_dev(double* b, int nrhs, int64_t ldb, bool wide = false) = 0;
    h2_factor_stats stats{};
    int64_t bytes_now = 0;
    int precision = H2_PREC_FP64;
    std::vector<double> norm_sys;             // ||A_s|| of every system (caller order)
    cudaStream_t stream = nullptr;
    const MatrixObj* A = nullptr;
    std::vector<std::vector<int64_t>> lay_sizes, lay_ranks, lay_rowptr, lay_col, lay_offset;
    std::vector<std::vector<int32_t>> lay_colour, lay_kind;
};

std::unique_ptr<FactorBase> make_factor(const MatrixObj* A, const h2_factor_opts& o);

template <class T>
struct FactorImpl : FactorBase {
    double eps_lu = 0, norm_a = 0;
    bool tensor_schur = false;                // H2_PREC_TF32X3: Schur update on tcgen05
    bool w_inverse = false;                   // D_RR^-1 formed explicitly (W_U, W_L, diagonal solve)
    std::vector<int> force;                   // debug: forced ranks of every level (concatenated)
    std::vector<int64_t> force_off;           // offset of each level in `force`
    std::vector<LevelRT> lv;
    // dense top matrices (float64), one per system
    int64_t nt = 0;                           // sum of their orders
    std::vector<int64_t> sys_nt, sys_xt;      // order, prefix of orders
    std::vector<DevBuf> sys_Dt, sys_piv;
    std::vector<TopSys> tops;
    DevBuf d_tops, d_sys_nt, d_sys_xt;
    DevBuf status;
    // events for phase timing
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_phase;
    std::vector<std::future<LevelCounts>> counts;   // per level, computed on worker threads
    // optional per-launch events (H2_FLAG_TIME_KERNELS)
    bool time_kernels = false;
    long long wait_budget = 4000000000LL;     // tensor-core Schur pipeline waits (SM cycles)
    int k_cap = 0;                            // cap on the augmented ranks (0: none)
    std::vector<cudaEvent_t> kev;
    std::vector<int> kev_id;
    void kbegin(int id);
    void kend();

    FactorImpl(const MatrixObj* A_, const h2_factor_opts& o);
    ~FactorImpl() override;
    void factorize() override;
    void solve_dev(double* b, int nrhs, int64_t ldb, bool wide = false) override;
    template <class V>
    void solve_in(double* b, int nrhs, int64_t ldb);

   private:
    void setup_level(size_t a);
    void run_level(size_t a);
    void close_level(size_t a);
    void assemble_tops(size_t a);
    void top_factor();
    void mark(int phase);
    void check_status(const char* where);
    void account(int phase, double flops, double bytes) {
        stats.phase_flops[phase] += flops;
        stats.phase_bytes[phase] += bytes;
    }
};

}  // namespace h2rs

struct h2_factor {
    std::unique_ptr<h2rs::FactorBase> f;
};
