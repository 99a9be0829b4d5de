// cs_smooth_noalloc: one application of a depth-nu cascade on a caller-given
// structured operator, with no device allocation anywhere on its path.
//
// The ping-pong vector that cs_smooth takes from its hierarchy handle lives
// here in a file-scope device array of fixed size, which every GPU that
// loads the library keeps until the process exits.  Host code cannot use
// the array's name as a device address (in host code it names a host-side
// shadow), so the address is fetched with cudaGetSymbolAddress once per
// device, the first time the entry point runs with that device current.
#include <mutex>

#include "cs_internal.cuh"

namespace csx {

constexpr int64_t NOALLOC_MAX_N = (int64_t)1 << 21;  // 2,097,152 doubles = 16 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_N];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

static cs_status noalloc_scratch(double **out) {
    int dev = 0;
    CSX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device ordinal %d beyond the %d supported by cs_smooth_noalloc", dev, NOALLOC_MAX_DEVICES);
        return CS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CS_OK;
}

// Every vector must be device (or managed) memory of the current device: the
// kernels and the scratch array run there, and a pointer into another GPU's
// memory (or into host memory) would be dereferenced without peer access.
static cs_status check_on_device(const void *ptr, const char *name) {
    int dev = 0;
    CSX_CUDA(cudaGetDevice(&dev));
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        set_error("%s is not a CUDA device pointer", name);
        return CS_ERR_ARG;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
        set_error("%s must be device memory of the current device %d (memory type %d, device %d)", name, dev,
                  (int)at.type, at.device);
        return CS_ERR_ARG;
    }
    return CS_OK;
}

}  // namespace csx

using namespace csx;

extern "C" cs_status cs_smooth_noalloc(int dim, const int *n, int box, const double *coeff, const double *lam,
                                       int nu, int kind, int reverse, const double *b, double *x,
                                       cs_stream stream) {
    if (!n || !coeff || !lam || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return CS_ERR_ARG; }
    if (n[0] < 1 || n[1] < 1 || (dim == 3 && n[2] < 1)) { set_error("bad grid size"); return CS_ERR_ARG; }
    if (nu < 1 || nu > 8) { set_error("nu must be in 1..8"); return CS_ERR_ARG; }
    if (kind != CS_ADDITIVE && kind != CS_MULTIPLICATIVE) { set_error("bad cascade kind"); return CS_ERR_ARG; }
    Level L;
    L.g = make_grid(dim, n[0], n[1], dim == 3 ? n[2] : 1);
    if (L.g.N > NOALLOC_MAX_N) {
        set_error("cs_smooth_noalloc handles at most %lld unknowns (got %lld)", (long long)NOALLOC_MAX_N,
                  (long long)L.g.N);
        return CS_ERR_ARG;
    }
    // the node kernels launch ceil(nx/TBX) x ceil(ny/TBY) x nz CTAs
    if ((int64_t)L.g.ny > (int64_t)TBY * 65535 || L.g.nz > 65535) {
        set_error("cs_smooth_noalloc: grid %d x %d x %d exceeds the launch limits (ny <= %d, nz <= 65535)", L.g.nx,
                  L.g.ny, L.g.nz, TBY * 65535);
        return CS_ERR_ARG;
    }
    L.kind = box ? BOX : STAR;
    L.nst = box ? (dim == 3 ? 27 : 9) : 2 * dim + 1;
    CSX_TRY(check_on_device(coeff, "coeff"));
    CSX_TRY(check_on_device(lam, "lam"));
    CSX_TRY(check_on_device(b, "b"));
    CSX_TRY(check_on_device(x, "x"));
    double *scratch = nullptr;
    CSX_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = L.g.N;
    const int ncol = kind == CS_MULTIPLICATIVE ? 2 : 1;
    // red-black is a graph colouring of a STAR stencil: those colour steps run in
    // place; every other step reads one buffer and writes the whole other one
    const bool inplace = kind == CS_MULTIPLICATIVE && !box;
    double *cur = x, *other = scratch;
    for (int step = 0; step < nu; ++step) {
        const int lv = reverse ? nu - 1 - step : step;
        for (int kk = 0; kk < ncol; ++kk) {
            const int colour = ncol == 2 ? (reverse ? ncol - 1 - kk : kk) : -1;
            if (inplace) {
                CSX_TRY(launch_sweep<double>(L, coeff, lam + (int64_t)lv * N, b, cur, cur, colour, false, s));
            } else {
                CSX_TRY(launch_sweep<double>(L, coeff, lam + (int64_t)lv * N, b, cur, other, colour, false, s));
                std::swap(cur, other);
            }
        }
    }
    if (cur != x) CSX_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    return CS_OK;
}
