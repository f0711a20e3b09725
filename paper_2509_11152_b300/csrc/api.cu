// C-ABI of the library: object lifetimes, argument checks, error codes.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "factor_impl.h"
#include "matvec.cuh"

// Krylov vectors per restarted flexible-GMRES cycle of the refinement
#ifndef H2_GMRES_RESTART
#define H2_GMRES_RESTART 30
#endif

namespace h2rs {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void DevBuf::alloc(size_t nbytes, cudaStream_t s) {
    release();
    stream = s;
    if (nbytes == 0) nbytes = 1;
    cudaError_t e = cudaMallocAsync(&ptr, nbytes, s);
    if (e == cudaErrorMemoryAllocation) {
        // the pool keeps freed memory reserved; give it back and try once more
        (void)cudaGetLastError();
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaStreamSynchronize(s) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
            cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocAsync(&ptr, nbytes, s);
    }
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        throw Error{H2_ERR_OOM, "device allocation of " + std::to_string(nbytes) +
                                    " bytes failed: " + cudaGetErrorString(e)};
    }
    bytes = nbytes;
}

void DevBuf::release() {
    if (ptr) {
        cudaFreeAsync(ptr, stream);
        ptr = nullptr;
        bytes = 0;
    }
}

static void keep_pool_memory() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}


template <class T>
static void upload_values(DevBuf& b, const T* p, int64_t n, bool on_dev, cudaStream_t s) {
    b.alloc(std::max<int64_t>(1, n) * sizeof(T), s);
    if (n > 0)
        H2_CUDA_CHECK(cudaMemcpyAsync(b.ptr, p, n * sizeof(T),
                                      on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

}  // namespace h2rs

using namespace h2rs;

extern "C" {

const char* h2_last_error(void) { return g_err.c_str(); }
int64_t h2_kernel_launch_count(void) { return g_launches.load(); }
const char* h2_version(void) { return "h2rs 0.1 (sm_103a)"; }

int h2_matrix_create_batch(int32_t nsys, const h2_matrix_desc* descs, h2_matrix** out) {
    if (!out) { set_error("null output pointer"); return H2_ERR_ARG; }
    *out = nullptr;
    h2_matrix* A = nullptr;
    int rc = guard([&] {
        H2_REQUIRE(nsys >= 1 && descs != nullptr, H2_ERR_ARG, "need at least one descriptor");
        keep_pool_memory();
        A = new h2_matrix();
        MatrixObj& M = A->m;
        std::vector<HostStructure> parts(nsys);
        for (int z = 0; z < nsys; ++z) {
            read_structure(&descs[z], parts[z]);
            const HostStructure& p = parts[z];
            const h2_matrix_desc& d = descs[z];
            H2_REQUIRE((d.U || p.U_off.back() == 0) && (d.E || p.E_off.back() == 0) &&
                           (d.S || p.S_off.back() == 0) && (d.D || p.D_off.back() == 0),
                       H2_ERR_ARG, "null value array");
        }
        std::vector<int> order;
        ForestValues fv;
        merge_forest(parts, M.H, order, fv);
        parts.clear();
        M.stream = static_cast<cudaStream_t>(descs[0].stream);
        H2_CUDA_CHECK(cudaGetDevice(&M.device));
        cudaStream_t s = M.stream;
        const HostStructure& H = M.H;
        const int64_t nn = H.nnodes, nleaf = H.lev_cnt[H.d];
        auto place = [&](DevBuf& b, int64_t total, const std::vector<ValueChunk>& ch, auto member) {
            b.alloc(std::max<int64_t>(1, total) * sizeof(double), s);
            for (const ValueChunk& c : ch) {
                const h2_matrix_desc& d = descs[c.sys];
                const double* src = d.*member;
                H2_CUDA_CHECK(cudaMemcpyAsync(b.as<double>() + c.dst, src + c.src, c.cnt * sizeof(double),
                                              d.values_on_device ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice, s));
            }
        };
        place(M.U, H.U_off[nleaf], fv.U, &h2_matrix_desc::U);
        place(M.E, H.E_off[nn], fv.E, &h2_matrix_desc::E);
        place(M.S, H.S_off.back(), fv.S, &h2_matrix_desc::S);
        place(M.D, H.D_off.back(), fv.D, &h2_matrix_desc::D);
        // the level plan is host work: build it while the value copies above are in
        // flight (from pinned host memory they run asynchronously), before the small
        // uploads below, whose pageable sources may make them wait for those copies
        build_plan(H, M.plan);
        upload(M.d_node_start, H.node_start, s);
        upload(M.d_node_size, H.node_size, s);
        upload(M.d_rank, H.rank, s);
        upload(M.d_U_off, H.U_off, s);
        upload(M.d_E_off, H.E_off, s);
        upload(M.d_S_off, H.S_off, s);
        upload(M.d_D_off, H.D_off, s);
        upload(M.d_adm_ptr, H.adm_ptr, s);
        upload(M.d_adm_col, H.adm_col, s);
        upload(M.d_inad_ptr, H.inad_ptr, s);
        upload(M.d_inad_col, H.inad_col, s);
        upload(M.d_parent, H.parent, s);
        std::vector<int64_t> child0(nn, -1);
        for (int l = 0; l < H.d; ++l)
            for (int64_t i = 0; i < H.lev_cnt[l]; ++i) child0[H.lev_first[l] + i] = H.lev_first[l + 1] + 2 * i;
        upload(M.d_child0, child0, s);
        upload(M.d_sys_voff, H.sys_voff, s);
        M.coef_off.assign(nn + 1, 0);
        for (int64_t g = 0; g < nn; ++g) M.coef_off[g + 1] = M.coef_off[g] + H.rank[g];
        upload(M.d_coef_off, M.coef_off, s);
        upload_plan(M.plan, s);
        H2_CUDA_CHECK(cudaStreamSynchronize(s));
    });
    if (rc != H2_OK) {
        // no copy may still read the caller's arrays once this returns
        if (nsys >= 1 && descs) cudaStreamSynchronize(static_cast<cudaStream_t>(descs[0].stream));
        delete A;
        return rc;
    }
    *out = A;
    return H2_OK;
}

int h2_matrix_create(const h2_matrix_desc* desc, h2_matrix** out) {
    if (!desc) {
        if (out) *out = nullptr;
        set_error("null descriptor");
        return H2_ERR_ARG;
    }
    return h2_matrix_create_batch(1, desc, out);
}

int h2_matrix_batch_info(const h2_matrix* A, int32_t* nsys, int64_t* sys_offset) {
    if (!A) { set_error("null matrix"); return H2_ERR_ARG; }
    const HostStructure& H = A->m.H;
    if (nsys) *nsys = H.nsys;
    if (sys_offset) for (int z = 0; z <= H.nsys; ++z) sys_offset[z] = H.sys_voff[z];
    return H2_OK;
}

void h2_matrix_destroy(h2_matrix* A) { delete A; }

int h2_matvec(const h2_matrix* A, int32_t nrhs, const double* x, int64_t ldx, double* y, int64_t ldy,
              int32_t on_device) {
    return guard([&] {
        H2_REQUIRE(A && x && y && nrhs > 0, H2_ERR_ARG, "bad matvec arguments");
        const MatrixObj& M = A->m;
        const int64_t n = M.H.n;
        H2_REQUIRE(ldx >= n && ldy >= n, H2_ERR_ARG, "leading dimension < n");
        cudaStream_t s = M.stream;
        if (on_device) {
            matvec_dev(M, nrhs, x, ldx, y, ldy, s);
        } else {
            DevBuf dx, dy;
            dx.alloc(n * nrhs * sizeof(double), s);
            dy.alloc(n * nrhs * sizeof(double), s);
            H2_CUDA_CHECK(cudaMemcpy2DAsync(dx.ptr, n * sizeof(double), x, ldx * sizeof(double),
                                            n * sizeof(double), nrhs, cudaMemcpyHostToDevice, s));
            matvec_dev(M, nrhs, dx.as<double>(), n, dy.as<double>(), n, s);
            H2_CUDA_CHECK(cudaMemcpy2DAsync(y, ldy * sizeof(double), dy.ptr, n * sizeof(double),
                                            n * sizeof(double), nrhs, cudaMemcpyDeviceToHost, s));
        }
        H2_CUDA_CHECK(cudaStreamSynchronize(s));
    });
}

int h2_factor_create(const h2_matrix* A, const h2_factor_opts* o, h2_factor** out) {
    if (!out) { set_error("null output pointer"); return H2_ERR_ARG; }
    *out = nullptr;
    h2_factor* Z = nullptr;
    int rc = guard([&] {
        H2_REQUIRE(A && o, H2_ERR_ARG, "null matrix or options");
        H2_REQUIRE(o->eps_lu >= 0 && std::isfinite(o->eps_lu), H2_ERR_ARG, "eps_lu must be >= 0");
        H2_REQUIRE((o->norm_a > 0 && std::isfinite(o->norm_a)) || o->sys_norm_a, H2_ERR_ARG,
                   "norm_a must be > 0");
        H2_REQUIRE(o->precision == H2_PREC_FP64 || o->precision == H2_PREC_FP32 ||
                       o->precision == H2_PREC_TF32X3,
                   H2_ERR_ARG, "unknown precision");
        Z = new h2_factor();
        Z->f = make_factor(&A->m, *o);
        Z->f->factorize();
    });
    if (rc != H2_OK) {
        delete Z;
        cudaStreamSynchronize(static_cast<cudaStream_t>(o ? o->stream : nullptr));
        return rc;
    }
    *out = Z;
    return H2_OK;
}

void h2_factor_destroy(h2_factor* Z) { delete Z; }

int h2_solve(const h2_factor* Z, int32_t nrhs, double* b, int64_t ldb, int32_t on_device) {
    return guard([&] {
        H2_REQUIRE(Z && b && nrhs > 0, H2_ERR_ARG, "bad solve arguments");
        FactorBase& F = *Z->f;
        const int64_t n = F.A->H.n;
        H2_REQUIRE(ldb >= n, H2_ERR_ARG, "ldb < n");
        cudaStream_t s = F.stream;
        if (on_device) {
            F.solve_dev(b, nrhs, ldb);
        } else {
            DevBuf db;
            db.alloc(n * nrhs * sizeof(double), s);
            H2_CUDA_CHECK(cudaMemcpy2DAsync(db.ptr, n * sizeof(double), b, ldb * sizeof(double),
                                            n * sizeof(double), nrhs, cudaMemcpyHostToDevice, s));
            F.solve_dev(db.as<double>(), nrhs, n);
            H2_CUDA_CHECK(cudaMemcpy2DAsync(b, ldb * sizeof(double), db.ptr, n * sizeof(double),
                                            n * sizeof(double), nrhs, cudaMemcpyDeviceToHost, s));
        }
        H2_CUDA_CHECK(cudaStreamSynchronize(s));
    });
}

int h2_refine_solve(const h2_factor* Z, const h2_matrix* A, int32_t nrhs, const double* b, int64_t ldb,
                    double* x, int64_t ldx, double tol, int32_t maxit, int32_t on_device, int32_t* iters,
                    double* berr) {
    int converged = 1;
    int rc = guard([&] {
        H2_REQUIRE(Z && A && b && x && nrhs > 0 && maxit >= 0, H2_ERR_ARG, "bad refine arguments");
        FactorBase& F = *Z->f;
        H2_REQUIRE(F.A == &A->m, H2_ERR_ARG, "factor belongs to another matrix");
        const int64_t n = A->m.H.n;
        H2_REQUIRE(ldb >= n && ldx >= n, H2_ERR_ARG, "leading dimension < n");
        cudaStream_t s = F.stream;
        DevBuf db, dx, dy, dr, dn;
        const double* bd = b;
        double* xd = x;
        int64_t lb = ldb, lx = ldx;
        const size_t vbytes = (size_t)n * nrhs * sizeof(double);
        if (!on_device) {
            db.alloc(vbytes, s);
            dx.alloc(vbytes, s);
            H2_CUDA_CHECK(cudaMemcpy2DAsync(db.ptr, n * sizeof(double), b, ldb * sizeof(double),
                                            n * sizeof(double), nrhs, cudaMemcpyHostToDevice, s));
            bd = db.as<double>();
            xd = dx.as<double>();
            lb = lx = n;
        }
        dy.alloc(vbytes, s);
        dr.alloc(vbytes, s);
        const HostStructure& HS = A->m.H;
        const int nseg = HS.nsys;
        dn.alloc(2 * (size_t)nseg * nrhs * sizeof(double), s);
        const int64_t* seg = A->m.d_sys_voff.as<int64_t>();
        H2_CUDA_CHECK(cudaMemcpy2DAsync(xd, lx * sizeof(double), bd, lb * sizeof(double), n * sizeof(double),
                                        nrhs, cudaMemcpyDeviceToDevice, s));
        F.solve_dev(xd, nrhs, lx);
        const std::vector<double>& nA = F.norm_sys;
        // channels q = c * nseg + z: column c of system z
        const int nq = nrhs * nseg;
        std::vector<double> h(2 * (size_t)nq), xscale(nq);
        // backward error of x (max over channels of ||r_q|| / (||A_z|| ||x_q||)); r = b - A x
        // is left in dr, and xscale[q] = ||A_z|| ||x_q||.
        auto residual = [&]() -> double {
            matvec_dev(A->m, nrhs, xd, lx, dy.as<double>(), n, s);
            residual_dev(bd, lb, dy.as<double>(), n, dr.as<double>(), n, n, nrhs, s);
            segnorm2_dev(dr.as<double>(), n, seg, nseg, nrhs, dn.as<double>(), s);
            segnorm2_dev(xd, lx, seg, nseg, nrhs, dn.as<double>() + nq, s);
            H2_CUDA_CHECK(cudaMemcpyAsync(h.data(), dn.ptr, 2 * (size_t)nq * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
            H2_CUDA_CHECK(cudaStreamSynchronize(s));
            double be = 0;
            for (int q = 0; q < nq; ++q) {
                const double r2 = h[q], x2 = h[nq + q];
                xscale[q] = nA[q % nseg] * std::sqrt(x2);
                const double e = xscale[q] > 0 ? std::sqrt(r2) / xscale[q] : (r2 > 0 ? INFINITY : 0.0);
                be = std::max(be, e);
            }
            H2_REQUIRE(std::isfinite(be), H2_ERR_NONFINITE, "non-finite residual in refinement");
            return be;
        };
        // One restarted flexible-GMRES cycle on A d = r, right-preconditioned by the
        // factor, classical Gram-Schmidt applied twice; float64.  The preconditioned
        // vectors z_j = M^-1 v_j are kept and d = Z y, so A Z = V H holds to float64
        // rounding and the cycle's residual estimate is the true residual.  M^-1 is
        // applied in float64 arithmetic over the stored factor (a fixed linear operator):
        // a float32 solve of an ill-conditioned system has rounding errors near
        // u_32 cond(A), which the Krylov space would have to absorb at every step.
        // Every channel (right-hand side of one system) has its own Krylov basis and
        // Hessenberg matrix, so a batch converges like its slowest system.  Used once
        // plain correction steps stop contracting (eps_lu * cond(A) near 1).
        DevBuf Vb, Zb, hb;
        auto gmres_cycle = [&](int m, double target_rel) -> int {
            Vb.alloc((size_t)(m + 1) * vbytes, s);
            Zb.alloc((size_t)m * vbytes, s);
            hb.alloc((size_t)(m + 1) * nq * sizeof(double), s);
            double* V = Vb.as<double>();
            double* hd = hb.as<double>();
            std::vector<double> beta(nq), sc(nq);
            segnorm2_dev(dr.as<double>(), n, seg, nseg, nrhs, dn.as<double>(), s);
            H2_CUDA_CHECK(cudaMemcpyAsync(h.data(), dn.ptr, nq * sizeof(double), cudaMemcpyDeviceToHost, s));
            H2_CUDA_CHECK(cudaStreamSynchronize(s));
            for (int q = 0; q < nq; ++q) {
                beta[q] = std::sqrt(h[q]);
                sc[q] = beta[q] > 0 ? 1.0 / beta[q] : 0.0;
            }
            H2_CUDA_CHECK(cudaMemcpyAsync(dn.ptr, sc.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s));
            scale_dev(dr.as<double>(), dn.as<double>(), n, nrhs, seg, nseg, V, s);
            std::vector<double> H((size_t)(m + 1) * m * nq, 0.0), g((size_t)(m + 1) * nq, 0.0),
                cs((size_t)m * nq), sn((size_t)m * nq), hh((size_t)(m + 1) * nq), h2((size_t)(m + 1) * nq);
            for (int q = 0; q < nq; ++q) g[q] = beta[q];
            auto Hc = [&](int row, int col, int q) -> double& { return H[((size_t)col * (m + 1) + row) * nq + q]; };
            int k = 0;
            for (int j = 0; j < m; ++j) {
                double* vj = V + (size_t)j * n * nrhs;
                double* w = V + (size_t)(j + 1) * n * nrhs;
                double* zj = Zb.as<double>() + (size_t)j * n * nrhs;
                H2_CUDA_CHECK(cudaMemcpyAsync(zj, vj, vbytes, cudaMemcpyDeviceToDevice, s));
                F.solve_dev(zj, nrhs, n, true);                              // z_j = M^-1 v_j
                matvec_dev(A->m, nrhs, zj, n, w, n, s);                       // A z_j
                for (int pass = 0; pass < 2; ++pass) {
                    multidot_dev(V, w, j + 1, n, nrhs, seg, nseg, hd, s);
                    H2_CUDA_CHECK(cudaMemcpyAsync(h2.data(), hd, (size_t)(j + 1) * nq * sizeof(double),
                                                  cudaMemcpyDeviceToHost, s));
                    H2_CUDA_CHECK(cudaStreamSynchronize(s));
                    for (size_t q = 0; q < (size_t)(j + 1) * nq; ++q) {
                        if (pass == 0) hh[q] = h2[q]; else hh[q] += h2[q];
                        h2[q] = -h2[q];
                    }
                    H2_CUDA_CHECK(cudaMemcpyAsync(hd, h2.data(), (size_t)(j + 1) * nq * sizeof(double),
                                                  cudaMemcpyHostToDevice, s));
                    combine_dev(V, hd, j + 1, n, nrhs, seg, nseg, w, s);
                }
                segnorm2_dev(w, n, seg, nseg, nrhs, dn.as<double>(), s);
                H2_CUDA_CHECK(cudaMemcpyAsync(h.data(), dn.ptr, nq * sizeof(double), cudaMemcpyDeviceToHost, s));
                H2_CUDA_CHECK(cudaStreamSynchronize(s));
                bool done = true;
                for (int q = 0; q < nq; ++q) {
                    const double hn = std::sqrt(h[q]);
                    sc[q] = hn > 0 ? 1.0 / hn : 0.0;
                    for (int i = 0; i <= j; ++i) Hc(i, j, q) = hh[(size_t)i * nq + q];
                    Hc(j + 1, j, q) = hn;
                    for (int i = 0; i < j; ++i) {                            // previous rotations
                        const double a0 = Hc(i, j, q), a1 = Hc(i + 1, j, q);
                        Hc(i, j, q) = cs[(size_t)i * nq + q] * a0 + sn[(size_t)i * nq + q] * a1;
                        Hc(i + 1, j, q) = -sn[(size_t)i * nq + q] * a0 + cs[(size_t)i * nq + q] * a1;
                    }
                    const double a0 = Hc(j, j, q), a1 = Hc(j + 1, j, q);
                    const double rr = std::hypot(a0, a1);
                    const double cj = rr > 0 ? a0 / rr : 1.0, sj = rr > 0 ? a1 / rr : 0.0;
                    cs[(size_t)j * nq + q] = cj;
                    sn[(size_t)j * nq + q] = sj;
                    Hc(j, j, q) = rr;
                    Hc(j + 1, j, q) = 0.0;
                    g[(size_t)(j + 1) * nq + q] = -sj * g[(size_t)j * nq + q];
                    g[(size_t)j * nq + q] = cj * g[(size_t)j * nq + q];
                    if (std::fabs(g[(size_t)(j + 1) * nq + q]) > target_rel * xscale[q]) done = false;
                }
                H2_CUDA_CHECK(cudaMemcpyAsync(dn.ptr, sc.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s));
                scale_dev(w, dn.as<double>(), n, nrhs, seg, nseg, w, s);
                k = j + 1;
                if (done) break;
            }
            // y = R^-1 g per channel; d = Z y (left in dr)
            std::vector<double> y((size_t)k * nq, 0.0);
            for (int q = 0; q < nq; ++q)
                for (int i = k - 1; i >= 0; --i) {
                    double t = g[(size_t)i * nq + q];
                    for (int p = i + 1; p < k; ++p) t -= Hc(i, p, q) * y[(size_t)p * nq + q];
                    y[(size_t)i * nq + q] = Hc(i, i, q) != 0 ? t / Hc(i, i, q) : 0.0;
                }
            H2_CUDA_CHECK(cudaMemcpyAsync(hd, y.data(), y.size() * sizeof(double), cudaMemcpyHostToDevice, s));
            H2_CUDA_CHECK(cudaMemsetAsync(dr.ptr, 0, vbytes, s));
            combine_dev(Zb.as<double>(), hd, k, n, nrhs, seg, nseg, dr.as<double>(), s);
            return k;
        };
        int it = 0;
        double be = residual(), prev = INFINITY;
        bool krylov = false;
        while (be > tol && it < maxit) {
            if (!krylov && be > 0.5 * prev) krylov = true;      // plain corrections stalled
            prev = be;
            if (!krylov) {
                F.solve_dev(dr.as<double>(), nrhs, n);
                ++it;
            } else {
                it += gmres_cycle(std::max(1, std::min(H2_GMRES_RESTART, maxit - it)), 0.5 * tol);
            }
            add_dev(xd, lx, dr.as<double>(), n, n, nrhs, s);
            be = residual();
        }
        if (!on_device)
            H2_CUDA_CHECK(cudaMemcpy2DAsync(x, ldx * sizeof(double), xd, n * sizeof(double), n * sizeof(double),
                                            nrhs, cudaMemcpyDeviceToHost, s));
        H2_CUDA_CHECK(cudaStreamSynchronize(s));
        if (iters) *iters = it;
        if (berr) *berr = be;
        converged = be <= tol;
    });
    if (rc != H2_OK) return rc;
    if (!converged) {
        set_error("refinement did not reach the tolerance");
        return H2_ERR_NO_CONVERGENCE;
    }
    return H2_OK;
}

int h2_factor_stats_get(const h2_factor* Z, h2_factor_stats* out) {
    if (!Z || !out) { set_error("null argument"); return H2_ERR_ARG; }
    *out = Z->f->stats;
    return H2_OK;
}

int h2_layout_counts(const h2_factor* Z, int32_t level, int64_t* nbox, int64_t* nblk) {
    if (!Z || level < 0 || level >= (int)Z->f->lay_sizes.size()) { set_error("bad level"); return H2_ERR_ARG; }
    if (nbox) *nbox = (int64_t)Z->f->lay_sizes[level].size();
    if (nblk) *nblk = (int64_t)Z->f->lay_col[level].size();
    return H2_OK;
}

int h2_layout_get(const h2_factor* Z, int32_t level, int64_t* sizes, int64_t* ranks, int32_t* colour,
                  int64_t* row_ptr, int64_t* col, int32_t* kind, int64_t* offset) {
    if (!Z || level < 0 || level >= (int)Z->f->lay_sizes.size()) { set_error("bad level"); return H2_ERR_ARG; }
    const FactorBase& F = *Z->f;
    auto cp = [](auto* dst, const auto& src) {
        if (dst) for (size_t q = 0; q < src.size(); ++q) dst[q] = src[q];
    };
    cp(sizes, F.lay_sizes[level]);
    cp(ranks, F.lay_ranks[level]);
    cp(colour, F.lay_colour[level]);
    cp(row_ptr, F.lay_rowptr[level]);
    cp(col, F.lay_col[level]);
    cp(kind, F.lay_kind[level]);
    cp(offset, F.lay_offset[level]);
    return H2_OK;
}

// host-only plan of a batch and the query of one of its levels (skeletonised levels
// only when only_skel)
static int plan_query_impl(int32_t nsys, const h2_matrix_desc* descs, int32_t level, bool only_skel,
                           int64_t* nbox, int64_t* nblk, int32_t* colour, int64_t* row_ptr, int64_t* col,
                           int32_t* kind, int32_t* state, int32_t* system) {
    return guard([&] {
        H2_REQUIRE(nsys >= 1 && descs != nullptr, H2_ERR_ARG, "need at least one descriptor");
        std::vector<HostStructure> parts(nsys);
        for (int z = 0; z < nsys; ++z) read_structure(&descs[z], parts[z]);
        HostStructure H;
        std::vector<int> order;
        ForestValues fv;
        merge_forest(parts, H, order, fv);
        Plan P;
        build_plan(H, P);
        const int nlev = (int)P.levels.size() + (only_skel ? 0 : 1);
        H2_REQUIRE(level >= 0 && level < nlev, H2_ERR_ARG, "bad level");
        const LevelStruct& S = level < (int)P.levels.size() ? P.levels[level] : P.toplev;
        if (nbox) *nbox = S.cnt;
        if (nblk) *nblk = S.nblocks();
        if (colour) for (int i = 0; i < S.cnt; ++i) colour[i] = S.colour[i];
        if (row_ptr) for (int i = 0; i <= S.cnt; ++i) row_ptr[i] = S.bptr[i];
        if (col) for (int b = 0; b < S.nblocks(); ++b) col[b] = S.bcol[b];
        if (kind) for (int b = 0; b < S.nblocks(); ++b) kind[b] = S.bkind[b];
        if (state) for (int i = 0; i < S.cnt; ++i) state[i] = S.state[i];
        if (system) for (int i = 0; i < S.cnt; ++i) system[i] = H.sys[S.first + i];
    });
}

int h2_plan_query_batch(int32_t nsys, const h2_matrix_desc* descs, int32_t level, int64_t* nbox,
                        int64_t* nblk, int32_t* colour, int64_t* row_ptr, int64_t* col, int32_t* kind,
                        int32_t* state, int32_t* system) {
    return plan_query_impl(nsys, descs, level, false, nbox, nblk, colour, row_ptr, col, kind, state, system);
}

int h2_plan_query(const h2_matrix_desc* desc, int32_t level, int64_t* nbox, int64_t* nblk,
                  int32_t* colour, int64_t* row_ptr, int64_t* col, int32_t* kind) {
    if (!desc) { set_error("null descriptor"); return H2_ERR_ARG; }
    return plan_query_impl(1, desc, level, true, nbox, nblk, colour, row_ptr, col, kind, nullptr, nullptr);
}

}  // extern "C"
