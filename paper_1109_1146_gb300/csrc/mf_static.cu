// Allocation-free cut extraction for 2D grids (mf_min_cut_2d_noalloc).
//
// Same kernels as the cut extraction at the end of mf_solve (cut2d.cu: residual
// bit masks, block-wise closure passes in one cooperative launch), but every
// scratch byte they need lives in one file-scope device array instead of
// memory from cudaMalloc.
// The array is part of the library image: each GPU that loads the library
// holds it until the process exits.
#include <cstdint>
#include <string>

#include "../../include/mf.h"
#include "mf_internal.cuh"

namespace {

constexpr size_t kCtrBytes = 256;                   // counter words (closure flags, pass count)
constexpr size_t kStaticScratchBytes = 8u << 20;    // 8 MiB in total

__device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

}  // namespace

extern "C" mf_status mf_min_cut_2d_noalloc(const int64_t dims[2], int connectivity, const int32_t *res,
                                           const int32_t *tres, const int32_t *exc, uint8_t *smin,
                                           uint8_t *smax, void *cuda_stream) {
    using namespace mf;
    if (!dims || !res || !tres || !exc || !smin || !smax) {
        set_static_error("mf_min_cut_2d_noalloc: null pointer argument");
        return MF_EINVAL;
    }
    if (connectivity != 4 && connectivity != 8) {
        set_static_error("mf_min_cut_2d_noalloc: connectivity must be 4 or 8");
        return MF_EINVAL;
    }
    const long long X = dims[0], Y = dims[1];
    if (X < 1 || Y < 1 || X * Y > (1ll << 31) - 1) {
        set_static_error("mf_min_cut_2d_noalloc: dims must be >= 1 and X*Y < 2^31");
        return MF_EINVAL;
    }
    Geom g{};
    g.X = (int)X;
    g.Y = (int)Y;
    g.Z = 1;
    g.n = X * Y;
    g.tx = g.ty = 64;
    g.tz = 1;
    g.sx = g.sy = 6;
    g.sz = 0;
    g.RX = (int)((X + 63) / 64);
    g.RY = (int)((Y + 63) / 64);
    g.RZ = 1;
    g.nreg = g.RX * g.RY;
    g.dinf = 1;
    const size_t need = kCtrBytes + cut2d_scratch_bytes(g, connectivity);
    if (need > kStaticScratchBytes) {
        set_static_error("mf_min_cut_2d_noalloc: grid needs " + std::to_string(need) +
                         " bytes of scratch, more than the static maximum of " +
                         std::to_string(kStaticScratchBytes) + " bytes");
        return MF_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_static_error(std::string("mf_min_cut_2d_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return MF_ECUDA;
    }
    // The array's host-side name is not a device address: ask the runtime for
    // the address of the current device's copy on every call (cheap; a cached
    // address would go stale if the module were reloaded, e.g. after
    // cudaDeviceReset).
    void *base = nullptr;
    e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess || !base) {
        set_static_error(std::string("mf_min_cut_2d_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return MF_ECUDA;
    }
    DevState st{};
    st.cap = const_cast<int *>(res);
    st.tcap = const_cast<int *>(tres);
    st.exc = const_cast<int *>(exc);
    st.ctr = (int *)base;  // the closure kernel clears the flag words it uses
    e = cut2d(connectivity, g, st, (unsigned char *)base + kCtrBytes, smin, smax, nullptr, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_static_error(std::string("mf_min_cut_2d_noalloc: ") + cudaGetErrorString(e));
        return MF_ECUDA;
    }
    return MF_OK;
}
