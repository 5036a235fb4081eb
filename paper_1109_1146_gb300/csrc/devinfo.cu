// Per-device launch facts: SM count, co-residency of cooperative kernels and
// the dynamic shared-memory opt-in of the large kernels.  Every value is
// looked up for the device that is current when it is first needed and
// cached per (kernel, device), so that launches size their grids from the
// GPU they run on and several host threads or devices can share the library.
#include <map>
#include <mutex>
#include <utility>

#include "mf_internal.cuh"

namespace mf {

namespace {
std::mutex g_mu;
std::map<int, int> g_sms;                                  // device -> SMs
std::map<std::pair<const void *, int>, int> g_coop;        // (kernel, device) -> co-resident blocks (threads, smem fixed per kernel)
std::map<std::pair<const void *, int>, int> g_smem_attr;   // (kernel, device) -> dynamic smem bytes already allowed
}  // namespace

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    g_sms[dev] = sms;
    return sms;
}

cudaError_t coop_max_blocks(const void *kernel, int threads, size_t smem, int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_coop.find({kernel, dev});
        if (it != g_coop.end()) {
            *out = it->second;
            return cudaSuccess;
        }
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    const int blocks = per_sm * device_sms();
    if (blocks <= 0) return cudaErrorCooperativeLaunchTooLarge;
    std::lock_guard<std::mutex> lk(g_mu);
    g_coop[{kernel, dev}] = blocks;
    *out = blocks;
    return cudaSuccess;
}

cudaError_t ensure_smem_attr(const void *kernel, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_smem_attr.find({kernel, dev});
    if (it != g_smem_attr.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    g_smem_attr[{kernel, dev}] = bytes;
    return cudaSuccess;
}

}  // namespace mf
