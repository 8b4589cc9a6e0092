// Internal declarations of the lattice-propagation library (not part of the ABI).
//
// Device layout (all per-site arrays share it):
//   ghost-padded planes of pitch_x * pitch_y sites, nz planes, C order
//   [z][py][px] with px = x + G, py = y + G for interior (x, y).  The G-wide
//   ghost bands in x and y hold copies of the periodic images (or zeros
//   across a wall); kernels keep them current by writing every updated site
//   to all of its images.  z has no ghosts: kernels wrap plane indices.
//   pitch_x is a multiple of 8 so every row starts on a 16-byte boundary for
//   FP32 / FP32x2 / BF16 arrays (required by TMA tensor maps).
//   Hop weights are 6 planes [k][site] (k = +x, -x, +y, -y, +z, -z), FP32 or
//   BF16; rotation factors are float2; the state is rho (float), m (float2)
//   and mu_a (float, per enabled axis), each double-buffered.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lpc3d.h"

namespace lpc {

constexpr int kMaxGhost = 8;
constexpr int kNumSums = 6;          // Mre, Mim, P, dMSD_x, dMSD_y, dMSD_z
constexpr int kMaxTB = 8;            // deepest temporal block

// Everything a step kernel needs about one lattice, passed by value.
struct LatticeView {
    int nx, ny, nz;
    // planes a step updates and sums over: [zlo, zhi).  A whole lattice has
    // zlo = 0, zhi = nz; a slab of a z-decomposed lattice holds one halo plane
    // on each side (planes 0 and nz - 1, read but never written by its
    // steps), so zlo = 1, zhi = nz - 1 and no plane index wraps.
    int zlo, zhi;
    int G, Xp, Yp;
    int per_x, per_y, per_z;
    int msd_axes;
    long long Np;                    // padded sites
    const float* rho_in;
    const float2* m_in;
    const float* mu_in[3];
    float* rho_out;
    float2* m_out;
    float* mu_out[3];
    const void* w;                   // [6][Np] float or bf16
    const float2* R;                 // [Np]
    // gather form of the static data (one-step TMA kernel), unpadded rows of
    // pitch Xs (a multiple of 64), Ns = Xs * ny * nz; null until first used
    const void* gwin;                // [6][Ns] in-weights win_k(x) = w_k(x - e_k), float or bf16
    const float* gs;                 // [Ns] stay weight 1 - sum_k w_k(x)
    const float2* gR;                // [Ns] rotation
    const void* gdm;                 // [3][Ns][2] (w_+a(x), w_-a(x)) for the MSD axes y, z, float or bf16
    // with the x pairs: [nz][tiles_x][nyp][2] (nyp = ny rounded up to 8) the x out-weights at the edges
    // of each 64-column tile, (w_-x of its first column, w_+x of its last
    // site); the other x out-weights are the in-weights of the neighbours
    const void* gdx;
    int Xs;
    long long Ns;
    // link form of the static data (plain lattices; one-step TMA kernel), null
    // unless used: [3][nz][ny1][Xs] signed link weights (ny1 = ny + 1 rows,
    // row 0 the image of row ny - 1), R in gR; link_a: alpha/6 as stored
    const void* lnk;
    const void* lnk_x0;              // [nz][ny] links entering column 0 from the left
    int ny1;
    float link_a;
    // reductions: per-block partials, completion counter, history
    double* partials;                // [levels][grid][kNumSums]
    unsigned int* counter;
    long long* step;                 // device step counter (index of the input state)
    double2* histM;                  // [1 + nreg][cap]: the totals, then each region
    double* histP;                   // [1 + nreg][cap]
    double* histD;                   // [1 + nreg][3][cap]
    long long cap;
    // region labels (null without regions): uint8 [nz][ny][Xr], Xr = roundup(nx, 64)
    const uint8_t* region;
    int nreg;
    int Xr;
    // tiling of the TMA-fed one-step kernel (0 = its heuristic): tile rows
    // (8, 12 or 16) and work items per CTA, which sets the z-chunk length
    int t1_ty, t1_ipc;
};

// Reservoir faces f = 2 a + side (side 0 below coordinate 0, side 1 above
// n_a - 1): the ghost sites just outside a face hold fixed values.  x and y
// faces use the ghost bands of the padded planes; z faces use a halo plane
// below or above the lattice's own planes (a lattice with a z reservoir holds
// nz + 2 planes, with zlo = 1, and its steps never write the halos).
struct ResFaces {
    int on[6];
    double F[6];
    float rho[6];
    float2 m[6];
    __host__ __device__ bool any() const { return on[0] || on[1] || on[2] || on[3] || on[4] || on[5]; }
    __host__ __device__ bool any_z() const { return on[4] || on[5]; }
};

// Deterministic sum helpers --------------------------------------------------

// FP32 butterfly over the 32 lanes; every lane ends with the same value.
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Load a weight (FP32 or BF16 plane) widened to float.
template <typename WT> __device__ __forceinline__ float ldw(const WT* p);
template <> __device__ __forceinline__ float ldw<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldw<__nv_bfloat16>(const __nv_bfloat16* p) {
    unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(static_cast<unsigned int>(u) << 16);
}

// The per-site update (shared by every kernel so that all schedules give
// bit-identical states).  win[k] is the weight of the hop along e_k into the
// site from its source y - e_k, nb*[k] the state at that source; wout the
// site's own out-weights.  Explicit _rn intrinsics forbid FMA contraction
// differences between kernels.
struct SiteIn {
    float wout[6];
    float win[6];
    float r[6];
    float2 m[6];
    float rc;
    float2 mc;
    float2 R;
};

__device__ __forceinline__ float stay_weight(const float* wout) {
    float t = __fadd_rn(wout[0], wout[1]);
    t = __fadd_rn(t, wout[2]);
    t = __fadd_rn(t, wout[3]);
    t = __fadd_rn(t, wout[4]);
    t = __fadd_rn(t, wout[5]);
    return __fsub_rn(1.0f, t);
}

__device__ __forceinline__ void site_rho_m(const SiteIn& q, float s, float& r_out, float2& m_out) {
    float r = __fmul_rn(s, q.rc);
    float ar = __fmul_rn(s, q.mc.x);
    float ai = __fmul_rn(s, q.mc.y);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        r = __fmaf_rn(q.win[k], q.r[k], r);
        ar = __fmaf_rn(q.win[k], q.m[k].x, ar);
        ai = __fmaf_rn(q.win[k], q.m[k].y, ai);
    }
    r_out = r;
    // rotation by the destination's phase: (R.x + i R.y)(ar + i ai)
    m_out.x = __fmaf_rn(q.R.x, ar, __fmul_rn(-q.R.y, ai));
    m_out.y = __fmaf_rn(q.R.x, ai, __fmul_rn(q.R.y, ar));
}

// The population part of site_rho_m alone (same operations in the same
// order, so the same bits): the equilibration phase propagates rho only.
__device__ __forceinline__ float site_rho(const float* win, const float* r, float rc, float s) {
    float v = __fmul_rn(s, rc);
#pragma unroll
    for (int k = 0; k < 6; ++k) v = __fmaf_rn(win[k], r[k], v);
    return v;
}

// The magnetisation part of site_rho_m alone (same operations in the same
// order): kernels that update the populations of two sites at once with
// pair_rho take the magnetisation of each site here.
__device__ __forceinline__ void site_m(const SiteIn& q, float s, float2& m_out) {
    float ar = __fmul_rn(s, q.mc.x);
    float ai = __fmul_rn(s, q.mc.y);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        ar = __fmaf_rn(q.win[k], q.m[k].x, ar);
        ai = __fmaf_rn(q.win[k], q.m[k].y, ai);
    }
    m_out.x = __fmaf_rn(q.R.x, ar, __fmul_rn(-q.R.y, ai));
    m_out.y = __fmaf_rn(q.R.x, ai, __fmul_rn(q.R.y, ar));
}

// Two neighbouring sites at once (.x and .y) with the paired FP32
// instructions of sm_100 and later: every element is rounded as the scalar
// _rn instruction rounds it, so these give the bits of stay_weight, site_rho
// and site_mu site by site, in half the instructions.
__device__ __forceinline__ float2 stay_weight2(const float2* wout) {
    float2 t = __fadd2_rn(wout[0], wout[1]);
    t = __fadd2_rn(t, wout[2]);
    t = __fadd2_rn(t, wout[3]);
    t = __fadd2_rn(t, wout[4]);
    t = __fadd2_rn(t, wout[5]);
    // 1 - t: the product -1 * t is exact, so the fused form rounds once, as
    // the subtraction does
    return __ffma2_rn(make_float2(-1.0f, -1.0f), t, make_float2(1.0f, 1.0f));
}
__device__ __forceinline__ float2 pair_rho(const float2* win, const float2* r, float2 rc, float2 s) {
    float2 v = __fmul2_rn(s, rc);
#pragma unroll
    for (int k = 0; k < 6; ++k) v = __ffma2_rn(win[k], r[k], v);
    return v;
}
__device__ __forceinline__ float2 pair_mu(const float2* win, const float2* r, const float2* mu_nb, float2 s,
                                          float2 mu_c, int a) {
    float2 u = __fmul2_rn(s, mu_c);
#pragma unroll
    for (int k = 0; k < 6; ++k) u = __ffma2_rn(win[k], mu_nb[k], u);
    u = __ffma2_rn(win[2 * a], r[2 * a], u);
    u = __ffma2_rn(make_float2(-win[2 * a + 1].x, -win[2 * a + 1].y), r[2 * a + 1], u);
    return u;
}

// First moment along axis a: mu'(y) = s mu(y) + sum_k win_k [mu_k + d_ka r_k].
__device__ __forceinline__ float site_mu(const float* win, const float* r, const float* mu_nb,
                                         float s, float mu_c, int a) {
    float u = __fmul_rn(s, mu_c);
#pragma unroll
    for (int k = 0; k < 6; ++k) u = __fmaf_rn(win[k], mu_nb[k], u);
    u = __fmaf_rn(win[2 * a], r[2 * a], u);             // hop along +a: displacement +1
    u = __fmaf_rn(-win[2 * a + 1], r[2 * a + 1], u);    // hop along -a: displacement -1
    return u;
}

// The same MSD increment summed over destinations: the hops into a site
// along +a and -a from its sources, win_+a (2 mu + rho) + win_-a (-2 mu + rho)
// at those sources (each link's term, attributed to its destination; over
// the lattice the same total where every link joins two lattice sites).
__device__ __forceinline__ float site_dmsd_in(const float* win, const float* r, const float* mu_nb, int a) {
    const float up = __fmaf_rn(2.0f, mu_nb[2 * a], r[2 * a]);
    const float dn = __fmaf_rn(-2.0f, mu_nb[2 * a + 1], r[2 * a + 1]);
    return __fmaf_rn(win[2 * a], up, __fmul_rn(win[2 * a + 1], dn));
}

// dMSD contribution of a site: 2 (w+a - w-a) mu + (w+a + w-a) rho.
__device__ __forceinline__ float site_dmsd(const float* wout, float mu_c, float rc, int a) {
    float u = __fsub_rn(wout[2 * a], wout[2 * a + 1]);
    float q = __fadd_rn(wout[2 * a], wout[2 * a + 1]);
    return __fmaf_rn(__fmul_rn(2.0f, u), mu_c, __fmul_rn(q, rc));
}

// The ghost images of a site on periodic axes, without the site's own
// interior position (which the caller stores itself, e.g. with a vector
// store): together with it, the positions store_images writes.  With
// nx, ny >= 2G a site has at most one image offset per axis (+n within G of
// the lower face, -n within G of the upper), so at most three images.
template <typename T>
__device__ __forceinline__ void store_ghost_images(T* base, const LatticeView& v, int x, int y, long long zoff,
                                                   T val) {
    const int G = v.G;
    if (v.nx >= 2 * G && v.ny >= 2 * G) {
        const int dx = !v.per_x ? 0 : x < G ? v.nx : (x >= v.nx - G ? -v.nx : 0);
        const int dy = !v.per_y ? 0 : y < G ? v.ny : (y >= v.ny - G ? -v.ny : 0);
        const long long p = zoff + (long long)(y + G) * v.Xp + (x + G);
        if (dx) base[p + dx] = val;
        if (dy) base[p + (long long)dy * v.Xp] = val;
        if (dx && dy) base[p + (long long)dy * v.Xp + dx] = val;
        return;
    }
    const int px0 = v.per_x ? (x + G) % v.nx : x + G;
    const int pxe = v.per_x ? v.nx + 2 * G : x + G + 1;
    const int py0 = v.per_y ? (y + G) % v.ny : y + G;
    const int pye = v.per_y ? v.ny + 2 * G : y + G + 1;
    for (int py = py0; py < pye; py += v.ny)
        for (int px = px0; px < pxe; px += v.nx)
            if (px != x + G || py != y + G) base[zoff + (long long)py * v.Xp + px] = val;
}

// Write a site value to its interior position and every ghost image.
template <typename T>
__device__ __forceinline__ void store_images(T* base, const LatticeView& v, int x, int y,
                                             long long zoff, T val) {
    const int G = v.G;
    base[zoff + (long long)(y + G) * v.Xp + (x + G)] = val;
    if (x >= G && x < v.nx - G && y >= G && y < v.ny - G) return;
    store_ghost_images(base, v, x, y, zoff, val);
}

// Final reduction of per-warp FP64 sums held in shared memory as
// smem[(level * NW + warp) * kNumSums + q]: each block combines its warps in
// a fixed order into per-block partials, and the last block to finish sums
// the partials in a fixed order (lanes stride over blocks, then an FP64
// butterfly) and writes the history entries of `levels` consecutive steps
// starting at *v.step.
template <int NW>
__device__ void block_finish_smem(const LatticeView& v, int levels, double* smem) {
    __syncthreads();
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < levels * kNumSums) {
        const int l = tid / kNumSums, q = tid % kNumSums;
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += smem[(l * NW + w) * kNumSums + q];
        v.partials[((long long)l * nblk + bid) * kNumSums + q] = s;
    }
    __threadfence();
    __shared__ unsigned int is_last;
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(v.counter, 1u) == (unsigned)nblk - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const long long n0 = *v.step;
    for (int job = warp; job < levels * kNumSums; job += NW) {
        const int l = job / kNumSums, q = job % kNumSums;
        double s = 0.0;
        for (int b = lane; b < nblk; b += 32) s += __ldcg(&v.partials[((long long)l * nblk + b) * kNumSums + q]);
        s = warp_sum_f64(s);
        if (lane == 0) {
            const long long n = n0 + l;            // input state index of this level
            if (q == 0) v.histM[n + 1].x = s;
            else if (q == 1) v.histM[n + 1].y = s;
            else if (q == 2) v.histP[n + 1] = s;
            else if (n >= 0 && (v.msd_axes >> (q - 3) & 1)) v.histD[(long long)(q - 3) * v.cap + n] = s;
        }
    }
    __syncthreads();
    if (tid == 0) {
        *v.step = n0 + levels;
        *v.counter = 0u;
    }
}

// The fixed-order reduction of items_finish, run by every thread of one
// block: the items' FP64 partials into the history entries of one step at
// *v.step (thread t adds items t, t + T, ... in order into scratch[q][t];
// warp q adds the T values lane-strided and by an FP64 butterfly), then
// *v.step advances.  The result depends on the items' partials only.
template <int NW>
__device__ void items_reduce(const LatticeView& v, int n_items, double* scratch) {
    const int T = NW * 32;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    double acc[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int b = tid; b < n_items; b += T) {
        const double* p = v.partials + (long long)b * kNumSums;
#pragma unroll
        for (int q = 0; q < kNumSums; ++q) acc[q] += __ldcg(p + q);
    }
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) scratch[q * T + tid] = acc[q];
    __syncthreads();
    const long long n = *v.step;
    for (int q = warp; q < kNumSums; q += NW) {
        double s = 0.0;
        for (int t = lane; t < T; t += 32) s += scratch[q * T + t];
        s = warp_sum_f64(s);
        if (lane == 0) {
            if (q == 0) v.histM[n + 1].x = s;
            else if (q == 1) v.histM[n + 1].y = s;
            else if (q == 2) v.histP[n + 1] = s;
            else if (n >= 0 && (v.msd_axes >> (q - 3) & 1)) v.histD[(long long)(q - 3) * v.cap + n] = s;
        }
    }
    __syncthreads();
    if (tid == 0) *v.step = n + 1;
}

// The arithmetic of items_reduce<NW> carried out by one warp, without a
// block-wide barrier: lane l plays the threads t = l, l + 32, ... of a block
// of T = NW * 32 threads (each adds its items t, t + T, ... in order), adds
// their sums in increasing t (the lane-strided second stage of
// items_reduce), and the warp ends with the same FP64 butterfly.  The same
// additions in the same order give the same history entries.
template <int NW>
__device__ void items_reduce_warp(const LatticeView& v, int n_items) {
    const int T = NW * 32;
    const int lane = threadIdx.x & 31;
    double s[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = lane; t < T; t += 32) {
        double acc[kNumSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = t; b < n_items; b += T) {
            const double* p = v.partials + (long long)b * kNumSums;
#pragma unroll
            for (int q = 0; q < kNumSums; ++q) acc[q] += __ldcg(p + q);
        }
#pragma unroll
        for (int q = 0; q < kNumSums; ++q) s[q] += acc[q];
    }
#pragma unroll
    for (int q = 0; q < kNumSums; ++q) s[q] = warp_sum_f64(s[q]);
    if (lane == 0) {
        const long long n = *v.step;
        v.histM[n + 1].x = s[0];
        v.histM[n + 1].y = s[1];
        v.histP[n + 1] = s[2];
        for (int q = 3; q < kNumSums; ++q)
            if (n >= 0 && (v.msd_axes >> (q - 3) & 1)) v.histD[(long long)(q - 3) * v.cap + n] = s[q];
        *v.step = n + 1;
    }
}

// Final reduction of per-item FP64 sums v.partials[item * kNumSums + q]
// written by the blocks of a work-queue kernel: the last block to finish
// runs items_reduce, so the result does not depend on which block took which
// item.  `scratch` is shared memory for kNumSums * blockDim doubles (free at
// this point).
template <int NW>
__device__ void items_finish(const LatticeView& v, int n_items, double* scratch) {
    const int tid = threadIdx.x;
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    __threadfence();
    __shared__ unsigned int is_last;
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(v.counter, 1u) == (unsigned)nblk - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    items_reduce<NW>(v, n_items, scratch);
    if (tid == 0) *v.counter = 0u;
}

// items_finish for items that also carry region sums: per item KS values,
// the kNumSums totals followed by kNumSums values for each of
// LPC_MAX_REGIONS regions (M_r and P_r of the output state, dMSD_r of the
// input state, like the totals); region r < v.nreg goes to history set 1 + r.
// The last block reads n_items * KS doubles: warp w takes a fixed contiguous
// chunk of items with lane q on value q (coalesced rows), spreading item j of
// the chunk over 16 accumulators (j mod 16) that are added in a fixed tree,
// then warp 0 adds the warps in order.  `scratch` holds 32 * NW doubles.
template <int NW, int KS>
__device__ void items_finish_regions(const LatticeView& v, int n_items, double* scratch) {
    static_assert(KS == kNumSums * (1 + LPC_MAX_REGIONS) && KS <= 32, "totals and every region slot");
    constexpr int A = 16;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    __threadfence();
    __shared__ unsigned int is_last_r;
    __syncthreads();
    if (tid == 0) is_last_r = (atomicAdd(v.counter, 1u) == (unsigned)nblk - 1u);
    __syncthreads();
    if (!is_last_r) return;
    __threadfence();
    const int chunk = (n_items + NW - 1) / NW;
    const int b0 = min(n_items, warp * chunk), b1 = min(n_items, b0 + chunk);
    double acc[A];
#pragma unroll
    for (int j = 0; j < A; ++j) acc[j] = 0.0;
    if (lane < KS) {
        const double* p = v.partials + lane;
        for (int b = b0; b < b1; b += A) {
#pragma unroll
            for (int j = 0; j < A; ++j)
                if (b + j < b1) acc[j] += __ldcg(p + (long long)(b + j) * KS);
        }
    }
#pragma unroll
    for (int w = A / 2; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) acc[j] += acc[j + w];
    scratch[warp * 32 + lane] = acc[0];
    __syncthreads();
    const long long n = *v.step;
    if (warp == 0 && lane < KS) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += scratch[w * 32 + lane];
        const int set = lane / kNumSums, qq = lane % kNumSums;
        if (set <= v.nreg) {
            if (qq == 0) v.histM[set * v.cap + n + 1].x = s;
            else if (qq == 1) v.histM[set * v.cap + n + 1].y = s;
            else if (qq == 2) v.histP[set * v.cap + n + 1] = s;
            else if (n >= 0 && (v.msd_axes >> (qq - 3) & 1))
                v.histD[((long long)set * 3 + (qq - 3)) * v.cap + n] = s;
        }
    }
    __syncthreads();
    if (tid == 0) {
        *v.step = n + 1;
        *v.counter = 0u;
    }
}

// Same, starting from per-warp sums in registers (lane 0 of every warp).
template <int NW>
__device__ void block_finish(const LatticeView& v, double (*acc)[kNumSums], int levels,
                             double* smem /* NW*kNumSums*levels */) {
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0)
        for (int l = 0; l < levels; ++l)
            for (int q = 0; q < kNumSums; ++q) smem[(l * NW + warp) * kNumSums + q] = acc[l][q];
    block_finish_smem<NW>(v, levels, smem);
}

// Host side --------------------------------------------------------------------

void set_error(const std::string& msg);
lpc_status cuda_fail(cudaError_t e, const char* what);

struct DeviceProps {
    int sm_count;
    int max_smem_optin;
};
const DeviceProps& device_props();

// Launchers (return cudaSuccess or the launch error).
// alpha_links: null (alpha on every link) or device [3][N] per-link factors.
// rf: reservoir faces (their out- and in-weights are packed beside the others).
// [z0, z1): the planes packed (z1 < 0: to the last); a plane's weights read
// the fields of the plane and of its z neighbours only.
cudaError_t launch_pack(const LatticeView& v, int wdtype, const double* F, const double* omega,
                        const uint8_t* solid, double alpha, const double* alpha_links, double dt, double kT,
                        const ResFaces& rf, cudaStream_t st, int z0 = 0, int z1 = -1);
// Write the reservoir values into the ghost sites of the reservoir faces, in
// both state buffers.
cudaError_t launch_reservoir_ghosts(const LatticeView& v, const ResFaces& rf, cudaStream_t st);
// Region-resolved sums of the current state (index *v.step): M_r, P_r and
// dMSD_a,r into the region histories (dmsd_only: dMSD_a,r alone); part:
// [region_blocks()][6 * LPC_MAX_REGIONS] doubles, done: a zeroed completion
// counter.
cudaError_t launch_region_sums(const LatticeView& v, int wdtype, double* part, unsigned int* done,
                               bool dmsd_only, cudaStream_t st);
int region_blocks();
cudaError_t launch_init_state(const LatticeView& v, const double* rho0_dev, int init_mode,
                              const double* F, const uint8_t* solid, double kT, double* scratch,
                              cudaStream_t st);
cudaError_t launch_sum_state(const LatticeView& v, cudaStream_t st);
cudaError_t launch_step1(const LatticeView& v, int wdtype, cudaStream_t st);
int step1_grid(const LatticeView& v, int wdtype);
cudaError_t launch_unpad(const void* src, int elem_bytes, const LatticeView& v, void* dst_dev,
                         cudaStream_t st);
cudaError_t launch_pad(const void* src_dev, int elem_bytes, const LatticeView& v, void* dst,
                       cudaStream_t st);
cudaError_t launch_weights_f32(const LatticeView& v, int wdtype, float* dst_dev, cudaStream_t st);
cudaError_t launch_maxdiff(const float* a, const float* b, const LatticeView& v, double* out2,
                           cudaStream_t st);

// Batched one-step launches over many lattices.
constexpr int kMaxBatch = 48;        // lattices per launch (kernel parameter space)
constexpr int kBatchCZ = 16;         // planes per work item in batched launches
struct BatchEntry {
    LatticeView v;
    int item0;                       // first global item of this lattice
    int n_items, tiles_x, tiles_y, cz;
    int steps;                       // steps of this lattice in a multi-step launch
};
struct BatchParams {
    int count;
    int total_items;
    BatchEntry e[kMaxBatch];
};
int batch_items(const LatticeView& v, int* tiles_x, int* tiles_y, int* cz);
cudaError_t launch_batch(const BatchParams& bp, int wdtype, int msd, cudaStream_t st);
// Persistent cooperative launch of `nsteps` steps (entries sorted by steps,
// descending); bar: a device word, zeroed by the launcher.
cudaError_t launch_batch_multi(const BatchParams& bp, int wdtype, int msd, int nsteps, unsigned int* bar,
                               cudaStream_t st);

// Temporally blocked kernel (K steps per launch, TMA-staged planes).
struct TBMaps;
bool tb_supported(const LatticeView& v, int wdtype, int K);
cudaError_t tb_prepare(int wdtype, int K, int msd);
bool tb_encode_maps(const LatticeView& v, int wdtype, int W, int H, TBMaps* maps);
bool tb_box_dims(const LatticeView& v, int wdtype, int K, int* W, int* H);
// err points into the lattice's counter block: err[0] is the error word,
// err[7] the one-step TMA kernel's work-queue counter (reset per launch).
// rho_only: propagate rho alone (m and mu untouched, M sums zero), the
// equilibration phase.
cudaError_t launch_tma1(const LatticeView& v, int wdtype, const TBMaps& maps, unsigned int* err,
                        cudaStream_t st, bool rho_only = false);
// The one-step TMA kernel takes the region sums itself for this lattice
// (labels staged with the static data); otherwise the separate region pass
// runs after it.
bool t1_fused_regions(const LatticeView& v, int wdtype);
cudaError_t t1_prepare(int wdtype, int msd);
bool t1_supported(const LatticeView& v, int wdtype);
// Tile rows the TMA-fed one-step kernel uses for this lattice (the caller's
// choice in v.t1_ty if its rings fit, else the heuristic's), and the default
// work items per CTA.
int t1_tile_rows(const LatticeView& v, int wdtype);
int t1_default_items_per_cta();
// Multi-lattice launches of the TMA-fed one-step kernel (serving): up to
// kMaxMulti lattices of one group (weight type, tile height, ghost width)
// step once in one launch, each with the states and sums of its own launch.
constexpr int kMaxMulti = 24;
bool t1_multi_member(const LatticeView& v, int wdtype);
int t1_multi_group(const LatticeView& v, int wdtype);
// maps[i]: the tensor maps of lattice i's current input buffer; words: the
// launch's work-queue counter (one device word, zeroed here before the
// launch); each lattice counts its stored items in its own counter word.
cudaError_t launch_tma1_multi(const LatticeView* views, const TBMaps* const* maps, int count, int wdtype,
                              unsigned int* words, cudaStream_t st);
bool t1_encode_maps(const LatticeView& v, int wdtype, TBMaps* maps);
int gather_pitch(int nx);
cudaError_t launch_gather_pack(const LatticeView& v, int wdtype, void* win, float* s, float2* R, void* dm, void* dx,
                               cudaStream_t st);
// Link form of a plain lattice's static data (v.Xs, v.ny1 set); bad / a_out:
// device words (a link that does not fit the form; alpha/6 as stored).
cudaError_t launch_link_pack(const LatticeView& v, int wdtype, void* L, void* X0, float2* Rl, double alpha,
                             unsigned int* bad, float* a_out, cudaStream_t st);
cudaError_t launch_tb(const LatticeView& v, int wdtype, int K, const TBMaps& maps, unsigned int* err,
                      cudaStream_t st);
int tb_grid(const LatticeView& v, int wdtype, int K);
size_t tb_maps_size();
TBMaps* tb_maps_new();
void tb_maps_delete(TBMaps* m);

}  // namespace lpc
