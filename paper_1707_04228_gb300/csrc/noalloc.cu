// Stress recovery whose peak reduction needs no device allocation.
//
// gl_stress accepts host or device arrays and allocates device staging
// buffers on every call.  Some callers cannot allow that: a host framework
// that has reserved nearly all device memory for its own caching pool (after
// the local factors, little is left), a latency-bound loop where cudaMalloc
// and cudaFree would synchronise the device and stall other streams, or a
// deployment whose device footprint must be fixed once the library is loaded.
// gl_stress_noalloc serves them: the caller passes device buffers for every
// input and output, and the only scratch -- the per-block partial maxima of
// the resin peak -- lives in the file-scope device array below.
#include <mutex>

#include "gl_internal.h"

namespace gl {

namespace {

// One slot per 256-element block of the peak reduction: 16,384 slots of 8 B
// (128 KB), held by every GPU that loads the library until the process
// exits; meshes of up to 16,384 x 256 = 4,194,304 elements fit.
constexpr int NOALLOC_SLOTS = 16384;
constexpr int NOALLOC_BLOCK = 256;
constexpr int64_t NOALLOC_MAX_ELEMS = (int64_t)NOALLOC_SLOTS * NOALLOC_BLOCK;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_peak_partials[NOALLOC_SLOTS];

// Device address of g_peak_partials on `device`, looked up by the first call
// on that device (with the device current) and cached.  In host code the name
// g_peak_partials is only a host-side stand-in for the symbol, never a device
// address, so it is not passed to kernels directly.
double *peak_scratch(int device) {
    static std::mutex mu;
    static double *addr[NOALLOC_MAX_DEVICES] = {nullptr};
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) fail(GL_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        int cur = -1;
        GL_CUDA(cudaGetDevice(&cur));
        if (cur != device) fail(GL_ERR_STATE, "peak scratch looked up with another device current");
        void *p = nullptr;
        GL_CUDA(cudaGetSymbolAddress(&p, g_peak_partials));
        addr[device] = static_cast<double *>(p);
    }
    return addr[device];
}

// partials[b] = max of v over the masked elements of block b, -1e300 when it
// has none (the empty value gl_stress reports too).  Every slot a call reads
// is written by that call first, so nothing has to start at zero.
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_peak_partial(const double *__restrict__ v,
                                                                const uint8_t *__restrict__ mask, int64_t n,
                                                                double *__restrict__ partials) {
    __shared__ double red[NOALLOC_BLOCK];
    const int64_t i = (int64_t)blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    red[threadIdx.x] = (i < n && mask[i]) ? v[i] : -1e300;
    __syncthreads();
    for (int o = NOALLOC_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(1024) k_peak_final(const double *__restrict__ partials, int nb,
                                                     double *__restrict__ out) {
    __shared__ double red[1024];
    double m = -1e300;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, partials[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// cuMemGetAddressRange of the driver API, reached through the runtime (the
// library links no driver library), looked up once.
using AddressRangeFn = int (*)(unsigned long long *base, size_t *size, unsigned long long ptr);

AddressRangeFn address_range_fn() {
    static std::once_flag once;
    static AddressRangeFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRangeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

void require_device_span(const void *p, size_t bytes, const char *what) {
    AddressRangeFn fn = address_range_fn();
    if (!fn) fail(GL_ERR_CUDA, "cuMemGetAddressRange is not available from the driver");
    unsigned long long base = 0;
    size_t size = 0;
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    if (fn(&base, &size, a) != 0)
        fail(GL_ERR_INVALID_ARG, std::string(what) + ": not inside a device allocation");
    if (a < base || a - base > size || size - (a - base) < bytes)
        fail(GL_ERR_INVALID_ARG, std::string(what) + ": the device allocation ends " +
                                     std::to_string(size - (a - base)) + " bytes after it, the call needs " +
                                     std::to_string(bytes));
}

void stress_noalloc(const MeshHost &m, int device, const double *X, const double *C, const double *psi_x,
                    const uint8_t *resin, const double *u, double *s33, double *t13, double *peak, cudaStream_t s) {
    if (m.n_elem > NOALLOC_MAX_ELEMS)
        fail(GL_ERR_INVALID_ARG, "gl_stress_noalloc: the mesh has " + std::to_string(m.n_elem) +
                                     " elements; its fixed scratch holds the peak reduction of at most 4,194,304");
    double *scratch = peak ? peak_scratch(device) : nullptr;
    launch_stress(m, X, C, psi_x, u, s33, t13, s);
    if (peak) {
        const int nb = (int)((m.n_elem + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
        k_peak_partial<<<nb, NOALLOC_BLOCK, 0, s>>>(s33, resin, m.n_elem, scratch);
        k_peak_final<<<1, 1024, 0, s>>>(scratch, nb, peak);
        GL_CUDA(cudaGetLastError());
    }
}

}  // namespace gl
