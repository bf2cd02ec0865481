// hrc_noalloc.cu -- the forward pass for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: a renderer's per-frame callback that
// runs under an engine-owned memory budget, code inside a host framework
// whose allocator must own every device byte, or a plugin loaded into a
// process that forbids new device allocations after start-up (cudaMalloc
// also synchronises the device, which a real-time frame loop cannot
// afford).  hrc_fluence_noalloc serves them: it runs the same kernels as
// hrc_fluence, but every intermediate buffer (the T_0..T_N and R_0..R_{N-1}
// levels of the four quadrant frames and the arc table) lives in one
// file-scope __device__ array of fixed size, so the call allocates nothing.
// The caller still passes the input and output buffers.
//
// The array exists on every GPU that loads this library, until the process
// exits: HRC_NOALLOC_SCRATCH_BYTES (about 20.4 MB) for grids of at most
// 128 x 128 pixels with at most 4 channels.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "hrc.h"
#include "hrc_internal.cuh"
#include "launch.h"

using namespace hrc;

namespace {

constexpr int kMaxSide = HRC_NOALLOC_MAX_SIDE;
constexpr int kMaxChannels = 4;
constexpr int kMaxLevels = 7;                     // ceil(log2(128))
constexpr size_t kArcFloatOff = 0;                // float A_n table, (1 << n) + j
constexpr size_t kArcDoubleOff = 1024;            // double copy (unused by fp32 kernels)
constexpr size_t kStatusOff = 3072;               // status word of the bounded copy waits
constexpr size_t kLevelsOff = 3328;               // first T level

constexpr size_t cx_align(size_t x) { return (x + 255) / 256 * 256; }

// Bytes of the fp32 layout of a side x side grid with C channels, levels
// starting at kLevelsOff (the layout of build_plan, written out for the
// largest accepted grid).
constexpr size_t layout_bytes(int side, int C) {
    int N = 0;
    while ((1 << N) < side) ++N;
    const size_t Vs = (size_t(side) + 31) / 32 * 32;
    size_t off = kLevelsOff;
    for (int q = 0; q < 4; ++q) {
        for (int n = 0; n <= N; ++n) {
            const size_t Un = (size_t(side) + (size_t(1) << n) - 1) >> n;
            off = cx_align(off + Un * ((size_t(1) << n) + 1) * Vs * (C * 4 + 4));
        }
        for (int n = 0; n < N; ++n) {
            const size_t Un = (size_t(side) + (size_t(1) << n) - 1) >> n;
            off = cx_align(off + Un * (size_t(1) << n) * C * Vs * 4);
        }
    }
    off = cx_align(off + 4 * (size_t(2) << N));
    off = cx_align(off + 8 * (size_t(2) << N));
    return off;
}

constexpr size_t kScratchBytes = layout_bytes(kMaxSide, kMaxChannels);
static_assert(kScratchBytes == HRC_NOALLOC_SCRATCH_BYTES, "hrc.h states the scratch size");
static_assert((size_t(2) << kMaxLevels) * 4 <= kArcDoubleOff - kArcFloatOff, "arc table fits");
static_assert((size_t(2) << kMaxLevels) * 8 <= kStatusOff - kArcDoubleOff, "arc table fits");
static_assert(kStatusOff + sizeof(int) <= kLevelsOff, "status word fits");

// The scratch itself.  Host code must never use this name as an address: on
// the host it is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_dev_ptr[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};
// test hook (hrc_noalloc_debug_wait): bytes the trace's copy barrier
// expects but never receives, and the bound of that wait
int g_extra_tx = 0;
long long g_limit_ns = 2000000000LL;
RayTable g_rays;
bool g_rays_ready = false;
thread_local std::string g_err;

hrc_status fail(hrc_status st, const std::string &msg) {
    g_err = "hrc_fluence_noalloc: " + msg;
    set_global_error(g_err.c_str());
    return st;
}

// Once per device, with that device current: resolve the device address of
// the scratch array, write the constant arc table (Eq. 13) into it and clear
// the status word.  The address is resolved again on every call (no
// allocation, no synchronisation); if it ever differs from the cached one
// (the device was reset and the library's module loaded anew), the set-up
// runs again.
hrc_status setup_device(int dev, char **base) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_rays_ready) {
        g_rays = make_ray_table();
        g_rays_ready = true;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail(HRC_ECUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    if (g_ready[dev] && g_dev_ptr[dev] != static_cast<char *>(p)) g_ready[dev] = false;
    if (!g_ready[dev]) {
        cudaError_t ep = prepare_device_once();
        if (ep != cudaSuccess) return fail(HRC_ECUDA, std::string("kernel set-up failed: ") + cudaGetErrorString(ep));
        float af[size_t(2) << kMaxLevels] = {};
        double ad[size_t(2) << kMaxLevels] = {};
        for (int n = 0; n <= kMaxLevels; ++n) {
            const double s = double(1 << n);
            for (int j = 0; j < (1 << n); ++j) {
                const double a = std::atan2(2.0 * (j + 1) - s, s) - std::atan2(2.0 * j - s, s);
                ad[(size_t(1) << n) + j] = a;
                af[(size_t(1) << n) + j] = (float)a;
            }
        }
        char *d = static_cast<char *>(p);
        e = cudaMemcpy(d + kArcFloatOff, af, sizeof(af), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + kArcDoubleOff, ad, sizeof(ad), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(d + kStatusOff, 0, sizeof(int));
        if (e != cudaSuccess) return fail(HRC_ECUDA, std::string("arc table upload failed: ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = d;
        g_ready[dev] = true;
    }
    *base = g_dev_ptr[dev];
    return HRC_OK;
}

}  // namespace

extern "C" hrc_status hrc_fluence_noalloc(int W, int H, int channels, const float *emission,
                                          const float *sigma_t, float *out, void *cuda_stream) {
    if (W < 1 || H < 1 || W > kMaxSide || H > kMaxSide)
        return fail(HRC_EINVAL, "W and H must be in [1, " + std::to_string(kMaxSide) + "] (got " +
                                    std::to_string(W) + " x " + std::to_string(H) + ")");
    if (channels < 1 || channels > kMaxChannels) return fail(HRC_EINVAL, "channels must be in [1, 4]");
    if (!emission || !sigma_t || !out) return fail(HRC_EINVAL, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(emission) | reinterpret_cast<uintptr_t>(sigma_t) |
         reinterpret_cast<uintptr_t>(out)) & 15u)
        return fail(HRC_EINVAL, "pointers must be 16-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(HRC_ECUDA, "no usable current device");
    char *base = nullptr;
    hrc_status st = setup_device(dev, &base);
    if (st != HRC_OK) return st;
    Plan pl;
    const size_t end = build_plan(W, H, channels, 0, P_FP32, kLevelsOff, pl, /*adjoint=*/false);
    if (end > kScratchBytes) return fail(HRC_EINVAL, "grid does not fit the fixed scratch");
    pl.arena = base;
    pl.arcs_off = (long long)kArcFloatOff;
    pl.arcs_off_d = (long long)kArcDoubleOff;
    pl.status = reinterpret_cast<int *>(base + kStatusOff);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        pl.bulk_extra_tx = g_extra_tx;
        pl.bulk_limit_ns = g_limit_ns;
    }
    Recorder rec;   // timing off
    int launches = 0;
    e = launch_forward(pl, g_rays, emission, sigma_t, out, static_cast<cudaStream_t>(cuda_stream), &launches, &rec);
    if (e != cudaSuccess) return fail(HRC_ECUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return HRC_OK;
}

extern "C" hrc_status hrc_noalloc_sync(void *cuda_stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(HRC_ECUDA, "no usable current device");
    char *base = nullptr;
    hrc_status st = setup_device(dev, &base);
    if (st != HRC_OK) return st;
    e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, base + kStatusOff, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && status != 0) e = cudaMemset(base + kStatusOff, 0, sizeof(int));
    if (e != cudaSuccess) return fail(HRC_ECUDA, std::string("status read failed: ") + cudaGetErrorString(e));
    if (status == kWaitLost)
        return fail(HRC_ETIMEOUT, "a copy wait gave up and its copies did not land within the drain bound: "
                                  "results of later launches on this device are suspect");
    if (status != 0) return fail(HRC_ETIMEOUT, "a copy wait gave up: the last call's fluence is incomplete");
    return HRC_OK;
}

extern "C" hrc_status hrc_noalloc_debug_wait(int extra_bytes, long long limit_ns) {
    if (extra_bytes < 0 || extra_bytes > 4096) return fail(HRC_EINVAL, "extra_bytes must be in [0, 4096]");
    std::lock_guard<std::mutex> lock(g_mu);
    g_extra_tx = extra_bytes;
    g_limit_ns = limit_ns > 0 ? limit_ns : 2000000000LL;
    return HRC_OK;
}
