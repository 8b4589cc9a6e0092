// lpc_step_noalloc: one lattice time step that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocator) at
// the point where they advance the lattice.  Examples are host codes that
// reserve all device memory at start-up through their own pool and forbid
// allocation afterwards (an allocation in a time loop can synchronise the
// device or fail under memory pressure), and plain C hosts with no allocator
// hooks.  They pass their own device buffers for the inputs and outputs;
// the only scratch this step needs (per-plane partial sums and a completion
// counter) lives in a fixed array in this file.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents: each call clears the completion counter, and every plane
// partial is written before it is read.  Calls that overlap on the GPU (on
// different streams, or from different threads without ordering) race on the
// scratch and give wrong sums; order them.  The array is held by every GPU
// that loads this library until the process exits.
#include <cstdint>

#include "lpc_internal.cuh"

namespace lpc {

namespace {

constexpr int kNoAllocMaxPlanes = 4096;            // nz limit of lpc_step_noalloc
constexpr size_t kNoAllocScratchBytes = 256 + (size_t)kNoAllocMaxPlanes * 3 * sizeof(double);

// [0, 4): completion counter; [256, ...): per-plane FP64 sums (M re, M im, P)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Grid: one block per z plane.  Site arithmetic is the shared site_rho_m, so
// the state equals the library's own one-step kernel bit for bit.
__global__ void __launch_bounds__(256)
k_step_noalloc(int nx, int ny, int nz, int px, int py, int pz, const float* __restrict__ w,
               const float2* __restrict__ R, const float* __restrict__ rin, const float2* __restrict__ min_,
               float* __restrict__ rout, float2* __restrict__ mout, double* __restrict__ sums,
               unsigned char* scratch) {
    const long long N = (long long)nx * ny * nz;
    const int z = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
    double* plane_sums = reinterpret_cast<double*>(scratch + 256);
    __shared__ double wsum[8][3];
    double acc[3] = {0.0, 0.0, 0.0};
    const int zm = z == 0 ? (pz ? nz - 1 : -1) : z - 1;
    const int zp = z == nz - 1 ? (pz ? 0 : -1) : z + 1;
    const int segs = (nx + 31) / 32;
    for (int rs = warp; rs < ny * segs; rs += 8) {
        const int y = rs / segs;
        const int x = (rs % segs) * 32 + lane;
        float vr = 0.f, vi = 0.f, vp = 0.f;
        if (x < nx) {
            const long long i = ((long long)z * ny + y) * nx + x;
            // sources of the hops into i: -x side hops +x, +x side hops -x, ...
            long long src[6];
            src[0] = x > 0 ? i - 1 : (px ? i + nx - 1 : -1);
            src[1] = x < nx - 1 ? i + 1 : (px ? i - (nx - 1) : -1);
            src[2] = y > 0 ? i - nx : (py ? i + (long long)(ny - 1) * nx : -1);
            src[3] = y < ny - 1 ? i + nx : (py ? i - (long long)(ny - 1) * nx : -1);
            src[4] = zm >= 0 ? ((long long)zm * ny + y) * nx + x : -1;
            src[5] = zp >= 0 ? ((long long)zp * ny + y) * nx + x : -1;
            SiteIn q;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                q.wout[k] = __ldg(w + k * N + i);
                if (src[k] >= 0) {
                    q.win[k] = __ldg(w + k * N + src[k]);
                    q.r[k] = __ldg(rin + src[k]);
                    q.m[k] = __ldg(min_ + src[k]);
                } else {           // outside a wall: no hop
                    q.win[k] = 0.f;
                    q.r[k] = 0.f;
                    q.m[k] = make_float2(0.f, 0.f);
                }
            }
            q.rc = __ldg(rin + i);
            q.mc = __ldg(min_ + i);
            q.R = __ldg(R + i);
            float ro;
            float2 mo;
            site_rho_m(q, stay_weight(q.wout), ro, mo);
            rout[i] = ro;
            mout[i] = mo;
            vr = mo.x; vi = mo.y; vp = ro;
        }
        vr = warp_sum_f32(vr); vi = warp_sum_f32(vi); vp = warp_sum_f32(vp);
        if (lane == 0) { acc[0] += vr; acc[1] += vi; acc[2] += vp; }
    }
    if (lane == 0) { wsum[warp][0] = acc[0]; wsum[warp][1] = acc[1]; wsum[warp][2] = acc[2]; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += wsum[k][threadIdx.x];
        plane_sums[z * 3 + threadIdx.x] = s;
    }
    __threadfence();
    __shared__ unsigned int last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)nz - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 3) {              // planes in z order
        double s = 0.0;
        for (int k = 0; k < nz; ++k) s += __ldcg(&plane_sums[k * 3 + threadIdx.x]);
        sums[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Device address of the scratch array on the current device.  Looked up on
// every call (a host-side table lookup once the module is loaded), so the
// address stays valid after a cudaDeviceReset reloads the module; the first
// lookup on a device loads this library's device code there.
void* scratch_address(cudaError_t* err) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    return *err == cudaSuccess ? p : nullptr;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace
}  // namespace lpc

using namespace lpc;

extern "C" lpc_status lpc_step_noalloc(int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                                       const float* w, const float* R, const float* rho_in,
                                       const float* m_in, float* rho_out, float* m_out, double* sums,
                                       void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || !periodic) {
        set_error("lpc_step_noalloc: edges must be >= 1 and periodic non-NULL");
        return LPC_ERR_INVALID;
    }
    if (nz > kNoAllocMaxPlanes) {
        set_error("lpc_step_noalloc: nz exceeds the 4096-plane limit of its fixed scratch array");
        return LPC_ERR_INVALID;
    }
    if ((long long)nx * ny * nz > 2147483647LL) {
        set_error("lpc_step_noalloc: more than 2^31-1 sites");
        return LPC_ERR_INVALID;
    }
    for (int a = 0; a < 3; ++a)
        if (periodic[a] != 0 && periodic[a] != 1) {
            set_error("lpc_step_noalloc: periodic flags must be 0 or 1");
            return LPC_ERR_INVALID;
        }
    if (!w || !R || !rho_in || !m_in || !rho_out || !m_out || !sums) {
        set_error("lpc_step_noalloc: NULL buffer");
        return LPC_ERR_INVALID;
    }
    if (rho_in == rho_out || m_in == m_out) {
        set_error("lpc_step_noalloc: input and output buffers must differ");
        return LPC_ERR_INVALID;
    }
    // the kernel reads R and m as (re, im) float pairs and writes FP64 sums
    if (!aligned(R, 8) || !aligned(m_in, 8) || !aligned(m_out, 8) || !aligned(sums, 8) || !aligned(w, 4) ||
        !aligned(rho_in, 4) || !aligned(rho_out, 4)) {
        set_error("lpc_step_noalloc: R, m_in, m_out and sums must be 8-byte aligned, w, rho_in and rho_out "
                  "4-byte aligned");
        return LPC_ERR_INVALID;
    }
    cudaError_t e = cudaSuccess;
    void* scratch = scratch_address(&e);
    if (!scratch) return cuda_fail(e, "lpc_step_noalloc: cudaGetSymbolAddress");
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), st);      // the completion counter
    if (e != cudaSuccess) return cuda_fail(e, "lpc_step_noalloc: counter clear");
    k_step_noalloc<<<nz, 256, 0, st>>>(nx, ny, nz, periodic[0], periodic[1], periodic[2], w,
                                        reinterpret_cast<const float2*>(R), rho_in,
                                        reinterpret_cast<const float2*>(m_in), rho_out,
                                        reinterpret_cast<float2*>(m_out), sums,
                                        static_cast<unsigned char*>(scratch));
    e = cudaGetLastError();
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lpc_step_noalloc: launch");
}
