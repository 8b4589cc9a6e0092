// Region-resolved sums of the current state (the spectra and diffusion of
// separate parts of a system, e.g. bulk and electrodes, Sec. 4):
//   M_r(n) = sum of m(x, n), P_r(n) = sum of rho(x, n) and
//   dMSD_a,r(n) = sum of [2 (w_+a - w_-a) mu_a + (w_+a + w_-a) rho](x, n)
// over the sites x labelled r.  A separate pass after each step of the
// one-step kernels that do not reduce per region themselves.
//
// Deterministic: warps take 32-site row segments in a fixed assignment
// (segment s goes to global warp s mod (blocks * 8)); every lane adds its
// sites in FP32 over a run of 16 segments, then into FP64; warps combine by
// FP64 butterflies, blocks their warps in order, and the last block to finish
// adds the per-block partials in block order.  The result therefore depends
// on the lattice only, not on timing.
#include "lpc_internal.cuh"

namespace lpc {

namespace {

constexpr int kWarps = 8;
constexpr int kQ = 6;                           // Mre, Mim, P, dMSD x, y, z
constexpr int kRQ = LPC_MAX_REGIONS * kQ;       // values per block partial
constexpr int kFlush = 16;                      // segments summed in FP32

template <typename WT>
__global__ void __launch_bounds__(kWarps * 32) k_region_sums(LatticeView v, double* __restrict__ part,
                                                          unsigned int* __restrict__ done, int dmsd_only) {
    __shared__ double sm[kWarps][kRQ];
    __shared__ unsigned int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int segs = (v.nx + 31) / 32;
    const long long nseg = (long long)segs * v.ny * v.nz;
    const long long stride = (long long)gridDim.x * kWarps;
    const WT* W = static_cast<const WT*>(v.w);
    double acc[LPC_MAX_REGIONS][kQ];
    float fa[LPC_MAX_REGIONS][kQ];
#pragma unroll
    for (int r = 0; r < LPC_MAX_REGIONS; ++r)
#pragma unroll
        for (int q = 0; q < kQ; ++q) { acc[r][q] = 0.0; fa[r][q] = 0.0f; }
    int run = 0;
    for (long long sidx = (long long)blockIdx.x * kWarps + warp; sidx < nseg; sidx += stride) {
        const int seg = (int)(sidx % segs);
        const long long row = sidx / segs;
        const int y = (int)(row % v.ny);
        const int z = (int)(row / v.ny);
        const int x = seg * 32 + lane;
        if (x < v.nx) {
            const long long p = ((long long)z * v.Yp + y + v.G) * v.Xp + x + v.G;
            const int lab = v.region[((long long)z * v.ny + y) * v.Xr + x];
            const float2 m = v.m_in[p];
            const float rho = v.rho_in[p];
            float val[kQ] = {m.x, m.y, rho, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (!(v.msd_axes >> a & 1)) continue;
                float wo[6];
                wo[2 * a] = ldw<WT>(W + (long long)(2 * a) * v.Np + p);
                wo[2 * a + 1] = ldw<WT>(W + (long long)(2 * a + 1) * v.Np + p);
                val[3 + a] = site_dmsd(wo, v.mu_in[a][p], rho, a);
            }
#pragma unroll
            for (int r = 0; r < LPC_MAX_REGIONS; ++r)
#pragma unroll
                for (int q = 0; q < kQ; ++q) fa[r][q] = __fadd_rn(fa[r][q], lab == r ? val[q] : 0.0f);
        }
        if (++run == kFlush) {
            run = 0;
#pragma unroll
            for (int r = 0; r < LPC_MAX_REGIONS; ++r)
#pragma unroll
                for (int q = 0; q < kQ; ++q) { acc[r][q] += (double)fa[r][q]; fa[r][q] = 0.0f; }
        }
    }
#pragma unroll
    for (int r = 0; r < LPC_MAX_REGIONS; ++r)
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            double t = warp_sum_f64(acc[r][q] + (double)fa[r][q]);
            if (lane == 0) sm[warp][r * kQ + q] = t;
        }
    __syncthreads();
    const int tid = threadIdx.x;
    if (tid < kRQ) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sm[w][tid];
        part[(long long)blockIdx.x * kRQ + tid] = t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(done, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid < kRQ) {
        double t = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) t += __ldcg(&part[(long long)b * kRQ + tid]);
        const int r = tid / kQ, q = tid % kQ;
        const long long n = *v.step;
        if (r < v.nreg && n >= 0) {
            const long long set = 1 + r;
            if (q < 3 && dmsd_only) {
            } else if (q == 0) {
                v.histM[set * v.cap + n].x = t;
            } else if (q == 1) {
                v.histM[set * v.cap + n].y = t;
            } else if (q == 2) {
                v.histP[set * v.cap + n] = t;
            } else if (v.msd_axes >> (q - 3) & 1) {
                v.histD[(set * 3 + (q - 3)) * v.cap + n] = t;
            }
        }
    }
    __syncthreads();
    if (tid == 0) *done = 0u;
}

}  // namespace

int region_blocks() { return device_props().sm_count * 2; }

cudaError_t launch_region_sums(const LatticeView& v, int wdtype, double* part, unsigned int* done,
                               bool dmsd_only, cudaStream_t st) {
    if (v.nreg <= 0 || !v.region) return cudaSuccess;
    if (wdtype == LPC_WEIGHTS_BF16)
        k_region_sums<__nv_bfloat16><<<region_blocks(), kWarps * 32, 0, st>>>(v, part, done, dmsd_only);
    else
        k_region_sums<float><<<region_blocks(), kWarps * 32, 0, st>>>(v, part, done, dmsd_only);
    return cudaGetLastError();
}

}  // namespace lpc
