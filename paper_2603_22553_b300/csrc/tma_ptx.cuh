// PTX helpers for TMA-fed kernels (mbarrier waits, bulk tensor copies) and
// the tensor maps they read.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "lpc_internal.cuh"

namespace lpc {

// Tensor maps of one input buffer parity (kernel parameter, __grid_constant__).
// w, R: padded hop-weight planes and rotation (multi-step kernel); gwin, gs,
// gR, gdm, gdx: the gather-form static arrays (one-step kernel); glab: the region
// labels (uint8, same rows as the gather form); glnk1, glnk2: the link form
// (boxes of TY and TY + 1 rows).
struct TBMaps {
    CUtensorMap rho, m, mu[3], w, R, gwin, gs, gR, gdm, gdx, glab, glnk1, glnk2;
};

bool tma_encode(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
                const cuuint64_t* strides, const cuuint32_t* box);
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

namespace {

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz: bound of every wait
// suspend-time hint of one try_wait (ns): a waiting warp sleeps in the
// barrier instead of spinning on issue slots; the loop re-checks the bound
constexpr uint32_t kSuspendNs = 200000;

__device__ __forceinline__ uint32_t sa(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(sa(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z, int c) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(sa(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(sa(bar)), "r"(x), "r"(y), "r"(z), "r"(c)
        : "memory");
}

// Warm the tensor-map cache with a descriptor (a hint; kernel-parameter or
// constant memory, generic address).
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

template <typename WT> __device__ __forceinline__ float lds_w(const WT* p);
template <> __device__ __forceinline__ float lds_w<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float lds_w<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __uint_as_float(static_cast<unsigned int>(*reinterpret_cast<const unsigned short*>(p)) << 16);
}

}  // namespace
}  // namespace lpc
