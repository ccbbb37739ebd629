// trk_find_peaks_noalloc: the local-maximum peak finder for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc at all: code running where an allocation could
// block or fail at an unpredictable moment (a trigger path with a fixed latency budget,
// a process that hands out all device memory up front through its own pool, a plug-in
// that receives device buffers from a host framework and may not own any).  Such a caller
// cannot create a trk handle (trk_create allocates every pool), but it may already hold
// dense vote histograms.  This entry point runs the same two peak kernels as
// trk_reconstruct on them; the kernels' only scratch (the per-bin maximum count over
// (d0, cot, z0), 4 bytes per bin, a list of the bins that reach their box maximum, up to
// 8 bytes per bin, and its counter) lives in the static device arrays below, so nothing is
// allocated: not by this file, not by the CUDA runtime on its behalf, not by torch.
//
// Costs and limits of that choice:
//   * the arrays take 24 MiB of device memory on every GPU that loads the library, until
//     the process exits, whether or not this entry point is used;
//   * a histogram may have at most TRK_NOALLOC_MAX_BINS (2^21) bins;
//   * all calls share the arrays, so two calls whose work overlaps on the GPU (on
//     different streams, or from different host threads) race and corrupt each other's
//     results; serialize them.  The arrays keep the last call's contents; each call writes
//     every count it reads and clears the list counter (and the caller's candidate bits)
//     itself before use;
//   * the arrays' device addresses are looked up once per device and kept for the life of
//     the process: after cudaDeviceReset the entry point must not be called again.
// Several small histograms share one pass of the kernels (as many as fit in the arrays, at
// most kMaxGroup); the bins the tie pass reads carry the event index.
#include <cstring>
#include <mutex>
#include <string>

#include "trk_common.cuh"

namespace trk {
size_t peak_pass1_smem(const FitConst &C, int td);
cudaError_t launch_peaks(const int32_t *hist, int32_t *m3, const FitConst &C, int g0, int G,
                         int td, int threshold, const int32_t *status, uint32_t *cbits, int64_t W,
                         uint32_t *filter, unsigned long long *ties, unsigned long long *n_ties,
                         int64_t tie_cap, int n_sm, cudaStream_t s, bool vec_ok);
cudaError_t launch_peak_ties(const int32_t *hist, const FitConst &C,
                             const unsigned long long *ties, const unsigned long long *n_ties,
                             int64_t tie_cap, uint32_t *cbits, int64_t W, uint32_t *filter,
                             unsigned long long *overflow, int n_sm, cudaStream_t s);
cudaError_t prepare_pipeline_kernels();
void set_global_error(const std::string &msg);
}  // namespace trk

using namespace trk;

// The peak finder's scratch, shared by every call on a device: per-bin box maxima, the
// list of bins that reach them (at most every bin), and [0] the list length, [1] a flag
// set when it would overflow (impossible below TRK_NOALLOC_MAX_BINS bins).
static __device__ __align__(256) int32_t g_peak_scratch[TRK_NOALLOC_MAX_BINS];
static __device__ __align__(256) unsigned long long g_peak_ties[TRK_NOALLOC_MAX_BINS];
static __device__ __align__(256) unsigned long long g_peak_counters[2];
// Per-event status read by the peak kernels: always zero (never written).
constexpr int kMaxGroup = 256;
static __device__ __align__(256) int32_t g_zero_status[kMaxGroup];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    int32_t *scratch = nullptr;    // device address of g_peak_scratch
    unsigned long long *ties = nullptr;      // g_peak_ties
    unsigned long long *counters = nullptr;  // g_peak_counters
    int32_t *zero = nullptr;       // device address of g_zero_status
    int n_sm = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

int noalloc_fail(int code, const std::string &msg)
{
    set_global_error(msg);
    return code;
}

// Once per device, with that device current: the device addresses of the static arrays
// (host code only sees host-side stand-ins for their names) and the kernels' shared-memory
// limit.
int setup_device(int dev, DeviceSetup **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(TRK_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_peak_scratch);
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                                  cudaGetErrorString(e));
        d.scratch = static_cast<int32_t *>(p);
        e = cudaGetSymbolAddress(&p, g_peak_ties);
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("cudaGetSymbolAddress(ties): ") +
                                                  cudaGetErrorString(e));
        d.ties = static_cast<unsigned long long *>(p);
        e = cudaGetSymbolAddress(&p, g_peak_counters);
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("cudaGetSymbolAddress(counters): ") +
                                                  cudaGetErrorString(e));
        d.counters = static_cast<unsigned long long *>(p);
        e = cudaGetSymbolAddress(&p, g_zero_status);
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("cudaGetSymbolAddress(status): ") +
                                                  cudaGetErrorString(e));
        d.zero = static_cast<int32_t *>(p);
        e = prepare_pipeline_kernels();
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("kernel attributes: ") +
                                                  cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || d.n_sm < 1)
            return noalloc_fail(TRK_ERR_CUDA, "multiprocessor count unavailable");
        d.ready = true;
    }
    *out = &d;
    return TRK_OK;
}

}  // namespace

extern "C" int trk_find_peaks_noalloc(const int32_t *hist, int32_t n_events,
                                      const trk_binning *binning, uint32_t *cand_bits,
                                      void *stream)
{
    if (!hist || !binning || !cand_bits || n_events < 1)
        return noalloc_fail(TRK_ERR_INVALID, "null pointer or n_events < 1");
    if (((uintptr_t)hist & 3) != 0 || ((uintptr_t)cand_bits & 3) != 0)
        return noalloc_fail(TRK_ERR_INVALID, "hist and cand_bits must be 4-byte aligned");
    double nb = 1.0;
    for (int k = 0; k < 5; ++k) {
        if (binning->n[k] < 1 || !(binning->lo[k] < binning->hi[k]))
            return noalloc_fail(TRK_ERR_INVALID, "invalid binning dimension");
        nb *= binning->n[k];
    }
    if (nb > (double)TRK_NOALLOC_MAX_BINS)
        return noalloc_fail(TRK_ERR_INVALID,
                            "histogram larger than TRK_NOALLOC_MAX_BINS (2^21 bins): use a "
                            "trk handle (trk_reconstruct), whose scratch is allocated");
    if (binning->periodic & ~1)
        return noalloc_fail(TRK_ERR_INVALID, "only dimension 0 (phi0) may be periodic");
    if (binning->threshold < 1)
        return noalloc_fail(TRK_ERR_INVALID, "threshold must be >= 1");
    if ((double)binning->n[3] * (binning->n[4] + 1) * 8.0 * 3.0 > 200.0 * 1024.0)
        return noalloc_fail(TRK_ERR_INVALID, "n[3] * (n[4] + 1) too large for the filter tile");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return noalloc_fail(TRK_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    DeviceSetup *d = nullptr;
    const int rc = setup_device(dev, &d);
    if (rc != TRK_OK)
        return rc;

    // the bin layout the peak kernels read (the rest of FitConst is unused by them)
    FitConst C;
    memset(&C, 0, sizeof(C));
    uint32_t stride = 1;
    for (int k = 4; k >= 0; --k) {
        C.stride[k] = stride;
        stride *= (uint32_t)binning->n[k];
        C.n[k] = binning->n[k];
    }
    C.nbins = (uint32_t)nb;
    C.periodic = binning->periodic;
    const int64_t W = ((int64_t)C.nbins + 31) / 32;
    int td = binning->n[2];
    while (td > 1 && peak_pass1_smem(C, td) > 48 * 1024)
        --td;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(cand_bits, 0, sizeof(uint32_t) * (size_t)W * n_events, s);
    if (e != cudaSuccess)
        return noalloc_fail(TRK_ERR_CUDA, std::string("clearing cand_bits: ") +
                                              cudaGetErrorString(e));
    // events per pass: their box maxima must fit in the scratch array
    int group = (int)(TRK_NOALLOC_MAX_BINS / C.nbins);
    group = group < 1 ? 1 : (group > kMaxGroup ? kMaxGroup : group);
    for (int g0 = 0; g0 < n_events; g0 += group) {
        const int G = n_events - g0 < group ? n_events - g0 : group;
        const int32_t *hg = hist + (size_t)g0 * C.nbins;
        // the 16-byte loads of pass 2 need a 16-byte aligned histogram
        const bool vec_ok = ((uintptr_t)hg & 15) == 0;
        e = cudaMemsetAsync(d->counters, 0, 2 * sizeof(unsigned long long), s);
        if (e == cudaSuccess)
            e = launch_peaks(hg, d->scratch, C, 0, G, td, binning->threshold, d->zero,
                             cand_bits + (size_t)g0 * W, W, nullptr, d->ties, d->counters,
                             TRK_NOALLOC_MAX_BINS, d->n_sm, s, vec_ok);
        if (e == cudaSuccess)
            e = launch_peak_ties(hg, C, d->ties, d->counters, TRK_NOALLOC_MAX_BINS,
                                 cand_bits + (size_t)g0 * W, W, nullptr, d->counters + 1,
                                 d->n_sm, s);
        if (e != cudaSuccess)
            return noalloc_fail(TRK_ERR_CUDA, std::string("peak kernels: ") +
                                                  cudaGetErrorString(e));
    }
    return TRK_OK;
}
