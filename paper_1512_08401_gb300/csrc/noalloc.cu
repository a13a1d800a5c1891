// Forward wavelet transform that allocates nothing (wdb_dwt_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside another framework's
// memory pool with the CUDA allocator locked down, real-time paths where a cudaMalloc (and
// the device-wide synchronisation it may imply) is not allowed, and callers holding a
// capture or a lock that an allocation would break. For them the multi-level transform keeps
// its intermediate approximations in a file-scope device array instead of a buffer from
// cudaMalloc. The array is part of the library image: every GPU that loads the library holds
// it (kNoAllocScratch floats, 16 MiB) until the process exits.
#include <mutex>

#include "wdb_internal.h"

namespace {

// Intermediate approximations of the multi-level DWT: at most N/2 floats for an N-pixel image.
constexpr long long kNoAllocScratch = 4LL * 1024 * 1024;
static __device__ __align__(256) float g_dwt_scratch[kNoAllocScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array for the current device (looked up once per device, with that
// device current). In host code the array's name is only a host-side stand-in, never a
// device address.
wdb_status scratch_for_current_device(float** out) {
    int dev = 0;
    WDB_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return wdb::set_error(WDB_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dwt_scratch);
        if (e != cudaSuccess) return wdb::cuda_error(e, "cudaGetSymbolAddress(g_dwt_scratch)", __FILE__, __LINE__);
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return WDB_OK;
}

}  // namespace

extern "C" wdb_status wdb_dwt_noalloc(const float* img_dev, float* coef_dev, int n_rows, int n_cols,
                                      const char* wavelet, int levels, void* stream) {
    using namespace wdb;
    if (!img_dev || !coef_dev) return set_error(WDB_EINVAL, "NULL argument");
    Layout L;
    WDB_TRY(make_layout(n_rows, n_cols, levels, &L));
    Filters f;
    WDB_TRY(wavelet_filters(wavelet, &f));
    if (L.N / 2 + 1 > kNoAllocScratch)
        return set_error(WDB_EINVAL, "wdb_dwt_noalloc: %dx%d needs %lld scratch floats, the static array holds %lld "
                                     "(at most %lld pixels)",
                         n_rows, n_cols, L.N / 2 + 1, kNoAllocScratch, 2 * (kNoAllocScratch - 1));
    float* scratch = nullptr;
    WDB_TRY(scratch_for_current_device(&scratch));
    return dwt2<float>(img_dev, coef_dev, L, f, scratch, static_cast<cudaStream_t>(stream));
}
