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

// Device address of the array on device `dev`, looked up once per device with that
// device current.  (In host code `g_matvec_scratch` names a host-side stand-in, not
// device memory.)
static double* scratch_for_device(int dev) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static double* addr[kMaxDevices] = {};
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

// x and y must be memory the matrix's device can address as its own: device memory of
// that device, or managed memory.  Host memory (pageable, pinned or mapped) and other
// devices' memory are rejected here instead of reaching a kernel.
static void require_device_vector(const void* p, int dev, const char* name) {
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error{H2_ERR_ARG, std::string("h2_matvec_static: ") + name + " is not a CUDA pointer"};
    }
    const bool ok = (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
    H2_REQUIRE(ok, H2_ERR_ARG,
               std::string("h2_matvec_static: ") + name + " must be device memory of the matrix's device " +
                   std::to_string(dev));
}

}  // namespace h2rs

using namespace h2rs;

extern "C" int h2_matvec_static(const h2_matrix* A, int32_t nrhs, const double* x, int64_t ldx, double* y,
                                int64_t ldy) {
    return guard([&] {
        H2_REQUIRE(A && x && y && nrhs > 0, H2_ERR_ARG, "bad h2_matvec_static arguments");
        const MatrixObj& M = A->m;
        const int64_t n = M.H.n;
        H2_REQUIRE(ldx >= n && ldy >= n, H2_ERR_ARG, "leading dimension < n");
        const int64_t need = 2 * M.coef_off.back() * (int64_t)nrhs;
        H2_REQUIRE(need <= (int64_t)H2_MATVEC_STATIC_WORDS, H2_ERR_ARG,
                   "h2_matvec_static: 2 * sum(rank) * nrhs = " + std::to_string(need) +
                       " doubles exceeds the static scratch of " + std::to_string(H2_MATVEC_STATIC_WORDS) +
                       " (use h2_matvec, or fewer right-hand sides per call)");
        // the kernels run on the matrix's stream, which belongs to the device current
        // when the matrix was created; the scratch address is per device, so the
        // current device must be that one
        int cur = -1;
        H2_CUDA_CHECK(cudaGetDevice(&cur));
        H2_REQUIRE(cur == M.device, H2_ERR_ARG,
                   "h2_matvec_static: current device " + std::to_string(cur) + " is not the matrix's device " +
                       std::to_string(M.device));
        require_device_vector(x, M.device, "x");
        require_device_vector(y, M.device, "y");
        double* scratch = scratch_for_device(M.device);
        // every coefficient the kernels read is written first in the same call (the
        // upsweep overwrites x-hat, the coupling step overwrites y-hat before the
        // downsweep adds to it), so the previous call's contents need no clearing
        matvec_dev(M, nrhs, x, ldx, y, ldy, M.stream, scratch);
        H2_CUDA_CHECK(cudaStreamSynchronize(M.stream));
    });
}
