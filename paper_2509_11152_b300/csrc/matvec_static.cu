// h2_matvec_static: the H^2 matrix-vector product with no device allocation.
//
// Some callers must not allocate device memory while they run: a host application
// that hands the library a GPU whose memory it manages itself and forbids further
// cudaMalloc/cudaFree calls, or a latency-critical loop (an iterative solver calling
// the product thousands of times) that cannot afford an allocator call or the
// synchronisation a cudaFree implies.  For them the coefficient vectors of the product
// (2 * sum of ranks * nrhs doubles) live in one file-scope device array of
// H2_MATVEC_STATIC_WORDS doubles.  Every GPU that loads the library holds that array
// until the process exits.
#include <mutex>

#include "h2rs_internal.h"
#include "matvec.cuh"

namespace h2rs {

static __device__ __align__(256) double g_matvec_scratch[H2_MATVEC_STATIC_WORDS];

// Device address of the array, looked up once per device with that device current.
// (In host code `g_matvec_scratch` names a host-side stand-in, not device memory.)
static double* scratch_for_current_device() {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static double* addr[kMaxDevices] = {};
    int dev = 0;
    H2_CUDA_CHECK(cudaGetDevice(&dev));
    H2_REQUIRE(dev >= 0 && dev < kMaxDevices, H2_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
        if (e != cudaSuccess)
            throw Error{H2_ERR_CUDA, std::string("cudaGetSymbolAddress(static matvec scratch): ") +
                                         cudaGetErrorString(e)};
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

}  // namespace h2rs

using namespace h2rs;

extern "C" int h2_matvec_static(const h2_matrix* A, int32_t nrhs, const double* x, int64_t ldx, double* y,
                                int64_t ldy) {
    try {
        H2_REQUIRE(A && x && y && nrhs > 0, H2_ERR_ARG, "bad h2_matvec_static arguments");
        const MatrixObj& M = A->m;
        const int64_t n = M.H.n;
        H2_REQUIRE(ldx >= n && ldy >= n, H2_ERR_ARG, "leading dimension < n");
        const int64_t need = 2 * M.coef_off.back() * (int64_t)nrhs;
        H2_REQUIRE(need <= (int64_t)H2_MATVEC_STATIC_WORDS, H2_ERR_ARG,
                   "h2_matvec_static: 2 * sum(rank) * nrhs = " + std::to_string(need) +
                       " doubles exceeds the static scratch of " + std::to_string(H2_MATVEC_STATIC_WORDS) +
                       " (use h2_matvec, or fewer right-hand sides per call)");
        double* scratch = scratch_for_current_device();
        // every coefficient the kernels read is written first in the same call (the
        // upsweep overwrites x-hat, the coupling step overwrites y-hat before the
        // downsweep adds to it), so the previous call's contents need no clearing
        matvec_dev(M, nrhs, x, ldx, y, ldy, M.stream, scratch);
        H2_CUDA_CHECK(cudaStreamSynchronize(M.stream));
        return H2_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unknown error in h2_matvec_static");
        return H2_ERR_ARG;
    }
}
