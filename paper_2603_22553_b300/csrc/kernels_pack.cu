// Once-per-lattice kernels: hop-weight packing, state initialisation, the
// initial sums, and the layout conversions used by the query calls.
#include "lpc_internal.cuh"

namespace lpc {

namespace {

// Interior coordinate of a padded position along one axis, or -1 when the
// position lies outside a wall (or in the pitch padding).
__device__ __forceinline__ int unpad_coord(int p, int G, int n, int per) {
    int c = p - G;
    if (c >= 0 && c < n) return c;
    if (!per || p >= n + 2 * G) return -1;
    c %= n;
    return c < 0 ? c + n : c;
}

__device__ __forceinline__ long long nb_site(int x, int y, int z, int k, int nx, int ny, int nz,
                                             int px, int py, int pz) {
    int c[3] = {x, y, z};
    const int n[3] = {nx, ny, nz};
    const int per[3] = {px, py, pz};
    const int a = k >> 1;
    c[a] += (k & 1) ? -1 : 1;
    if (c[a] < 0 || c[a] >= n[a]) {
        if (!per[a]) return -1;
        c[a] = c[a] < 0 ? n[a] - 1 : 0;
    }
    return ((long long)c[2] * ny + c[1]) * nx + c[0];
}

template <typename WT> __device__ __forceinline__ WT round_weight(double w);
template <> __device__ __forceinline__ float round_weight<float>(double w) { return __double2float_rn(w); }
template <> __device__ __forceinline__ __nv_bfloat16 round_weight<__nv_bfloat16>(double w) {
    return __double2bfloat16(w);
}

// Hop weights of Eq. 1 (Metropolis) times alpha/6 (six equally likely
// attempts, jump factor of Eq. 7); zero towards solids and across walls.
// With per-link factors (position-dependent diffusivity, Sec. 2.1 after
// Eq. 7) the factor of the link between a site and its +a neighbour is
// links[a][site], the same for both directions of the link.
// Rotation R = exp(i omega dt) in FP64, rounded to FP32.
// Reservoir faces (Sec. 3.2 item 1): a boundary pore site's move out of the
// domain through a reservoir face is accepted against the reservoir's F; the
// ghost site just outside the face carries the weight of the move from the
// reservoir into its boundary neighbour (the only one of its weights any
// kernel reads), so that the kernels' gather needs no special case.
__device__ __forceinline__ double metropolis(double dE) { return dE > 0.0 ? exp(-dE) : 1.0; }

// Reservoir ghost of a padded position: the face (0..3) when the position is
// the ghost site just outside a reservoir face next to an interior row or
// column, with the boundary site (bx, by) it feeds and the direction k of
// that move; -1 otherwise.
__device__ __forceinline__ int reservoir_ghost(const LatticeView& v, const ResFaces& rf, int px, int py,
                                               int x, int y, int& bx, int& by, int& k) {
    bx = x;
    by = y;
    if (x < 0 && y >= 0) {
        if (px == v.G - 1 && rf.on[0]) { bx = 0; k = 0; return 0; }
        if (px == v.G + v.nx && rf.on[1]) { bx = v.nx - 1; k = 1; return 1; }
    } else if (y < 0 && x >= 0) {
        if (py == v.G - 1 && rf.on[2]) { by = 0; k = 2; return 2; }
        if (py == v.G + v.ny && rf.on[3]) { by = v.ny - 1; k = 3; return 3; }
    }
    return -1;
}

template <typename WT>
__global__ void k_pack(LatticeView v, const double* __restrict__ F, const double* __restrict__ omega,
                       const uint8_t* __restrict__ solid, double alpha, const double* __restrict__ links,
                       double dt, double kT, ResFaces rf, long long p0, long long p1) {
    const long long pidx = p0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pidx >= p1) return;
    WT* W = static_cast<WT*>(const_cast<void*>(v.w));
    float2* R = const_cast<float2*>(v.R);
    const int px = (int)(pidx % v.Xp);
    const long long t = pidx / v.Xp;
    const int py = (int)(t % v.Yp);
    const int z = (int)(t / v.Yp);
    const int x = unpad_coord(px, v.G, v.nx, v.per_x);
    const int y = unpad_coord(py, v.G, v.ny, v.per_y);
    double w[6] = {0, 0, 0, 0, 0, 0};
    float2 rot = make_float2(1.0f, 0.0f);
    // FP64 divisions are slow on this part: alpha / 6 once per thread, and no
    // division by kT = 1 (both give the same values as dividing every time)
    const double a6 = alpha / 6.0;
    const bool unit_kT = kT == 1.0;
    if (x >= 0 && y >= 0) {
        const long long i = ((long long)z * v.ny + y) * v.nx + x;
        if (!solid[i]) {
            const long long N = (long long)v.nx * v.ny * v.nz;
            for (int k = 0; k < 6; ++k) {
                const long long j = nb_site(x, y, z, k, v.nx, v.ny, v.nz, v.per_x, v.per_y, v.per_z);
                if (j < 0) {
                    // out through a face: +a hops leave by side 1, -a hops by side 0
                    const int f = 2 * (k >> 1) + ((k & 1) ? 0 : 1);
                    if (k < 4 && rf.on[f]) {
                        const double d = rf.F[f] - F[i];
                        w[k] = a6 * metropolis(unit_kT ? d : d / kT);
                    }
                    continue;
                }
                if (solid[j]) continue;
                const double d = F[j] - F[i];
                const double dE = unit_kT ? d : d / kT;
                w[k] = (links ? links[(long long)(k >> 1) * N + ((k & 1) ? j : i)] / 6.0 : a6) * metropolis(dE);
            }
        }
        double s, c;
        sincos(omega[i] * dt, &s, &c);
        rot = make_float2(__double2float_rn(c), __double2float_rn(s));
    } else {
        int bx, by, k;
        const int f = reservoir_ghost(v, rf, px, py, x, y, bx, by, k);
        if (f >= 0) {
            const long long i = ((long long)z * v.ny + by) * v.nx + bx;
            const double d = F[i] - rf.F[f];
            if (!solid[i]) w[k] = a6 * metropolis(unit_kT ? d : d / kT);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) W[k * v.Np + pidx] = round_weight<WT>(w[k]);
    R[pidx] = rot;
}

// Deterministic FP64 sums for the Boltzmann normalisation: per-block fixed
// order, then one block over the partials.
__global__ void k_boltz_partial(const double* __restrict__ F, const uint8_t* __restrict__ solid,
                                long long N, double kT, double* part) {
    __shared__ double sz[256];
    __shared__ double sn[256];
    double z = 0.0, n = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        if (!solid[i]) { z += exp(-F[i] / kT); n += 1.0; }
    sz[threadIdx.x] = z;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) { sz[threadIdx.x] += sz[threadIdx.x + o]; sn[threadIdx.x] += sn[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = sz[0]; part[2 * blockIdx.x + 1] = sn[0]; }
}

__global__ void k_boltz_final(double* part, int nblk) {
    if (threadIdx.x != 0) return;
    double z = 0.0, n = 0.0;
    for (int b = 0; b < nblk; ++b) { z += part[2 * b]; n += part[2 * b + 1]; }
    part[2 * nblk] = z;
    part[2 * nblk + 1] = n;
}

// rho(x, 0) from rho0 (FP64, interior order), 1 on pore sites, or Eq. 2.
// m = rho, mu = 0.  Every padded position gets the value of its interior
// preimage (0 outside walls and in the pitch padding).
__global__ void k_init(LatticeView v, const double* __restrict__ rho0, int mode,
                       const double* __restrict__ F, const uint8_t* __restrict__ solid, double kT,
                       const double* __restrict__ zsum /* [Z, npore] or null */) {
    const long long pidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pidx >= v.Np) return;
    const int px = (int)(pidx % v.Xp);
    const long long t = pidx / v.Xp;
    const int py = (int)(t % v.Yp);
    const int z = (int)(t / v.Yp);
    const int x = unpad_coord(px, v.G, v.nx, v.per_x);
    const int y = unpad_coord(py, v.G, v.ny, v.per_y);
    float r = 0.0f;
    if (x >= 0 && y >= 0) {
        const long long i = ((long long)z * v.ny + y) * v.nx + x;
        if (!solid[i]) {
            if (rho0) r = __double2float_rn(rho0[i]);
            else if (mode == LPC_INIT_BOLTZMANN) r = __double2float_rn(zsum[1] * exp(-F[i] / kT) / zsum[0]);
            else r = 1.0f;
        }
    }
    // Both halves of the double buffer get the same values, so that ghost
    // positions no kernel ever writes (across walls, pitch padding) hold
    // zeros in either buffer: a zero hop weight times a stale NaN would be NaN.
    v.rho_out[pidx] = r;
    v.m_out[pidx] = make_float2(r, 0.0f);
    const_cast<float*>(v.rho_in)[pidx] = r;
    const_cast<float2*>(v.m_in)[pidx] = make_float2(r, 0.0f);
    for (int a = 0; a < 3; ++a)
        if (v.msd_axes >> a & 1) {
            v.mu_out[a][pidx] = 0.0f;
            const_cast<float*>(v.mu_in[a])[pidx] = 0.0f;
        }
}

// Reservoir values into the reservoir ghost sites of both state buffers
// (first moment 0).
__global__ void k_reservoir_ghosts(LatticeView v, ResFaces rf) {
    const long long pidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pidx >= v.Np) return;
    const int px = (int)(pidx % v.Xp);
    const long long t = pidx / v.Xp;
    const int py = (int)(t % v.Yp);
    const int z = (int)(t / v.Yp);
    const int x = unpad_coord(px, v.G, v.nx, v.per_x);
    const int y = unpad_coord(py, v.G, v.ny, v.per_y);
    int bx, by, k;
    int f = reservoir_ghost(v, rf, px, py, x, y, bx, by, k);
    // a z reservoir fills its whole halo plane (ghost bands included)
    if (rf.any_z() && v.zlo > 0) {
        if (z == v.zlo - 1) f = rf.on[4] ? 4 : -1;
        else if (z == v.zhi) f = rf.on[5] ? 5 : -1;
    }
    if (f < 0) return;
    v.rho_out[pidx] = rf.rho[f];
    v.m_out[pidx] = rf.m[f];
    const_cast<float*>(v.rho_in)[pidx] = rf.rho[f];
    const_cast<float2*>(v.m_in)[pidx] = rf.m[f];
    for (int a = 0; a < 3; ++a)
        if (v.msd_axes >> a & 1) {
            v.mu_out[a][pidx] = 0.0f;
            const_cast<float*>(v.mu_in[a])[pidx] = 0.0f;
        }
}

// Sums of the current state (M, P) into history entry *step + 1, using the
// same row-butterfly structure as the step kernels.
__global__ void __launch_bounds__(256) k_sum_state(LatticeView v) {
    __shared__ double smem[8 * kNumSums];
    double acc[1][kNumSums] = {{0, 0, 0, 0, 0, 0}};
    const int lane = threadIdx.x;
    const int rows = v.ny * v.nz;
    const int segs = (v.nx + 31) / 32;
    const long long plane = (long long)v.Xp * v.Yp;
    for (long long r = (long long)blockIdx.x * 8 + threadIdx.y; r < (long long)rows * segs;
         r += (long long)gridDim.x * 8) {
        const int seg = (int)(r % segs);
        const int row = (int)(r / segs);
        const int y = row % v.ny, z = row / v.ny;
        const int x = seg * 32 + lane;
        float vr = 0.f, vi = 0.f, vp = 0.f;
        if (x < v.nx) {
            const long long i = z * plane + (long long)(y + v.G) * v.Xp + x + v.G;
            const float2 m = v.m_in[i];
            vr = m.x; vi = m.y; vp = v.rho_in[i];
        }
        vr = warp_sum_f32(vr); vi = warp_sum_f32(vi); vp = warp_sum_f32(vp);
        if (lane == 0) { acc[0][0] += vr; acc[0][1] += vi; acc[0][2] += vp; }
    }
    block_finish<8>(v, acc, 1, smem);
}

// Interior extraction: dst[i] = src[padded(i)] for elements of 4 or 8 bytes.
template <typename T>
__global__ void k_unpad(const T* __restrict__ src, LatticeView v, T* __restrict__ dst) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % v.nx);
        const long long t = i / v.nx;
        const int y = (int)(t % v.ny);
        const int z = (int)(t / v.ny);
        dst[i] = src[((long long)z * v.Yp + y + v.G) * v.Xp + x + v.G];
    }
}

// Interior scatter with ghost images (inverse of k_unpad).
template <typename T>
__global__ void k_pad(const T* __restrict__ src, LatticeView v, T* __restrict__ dst) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    const long long plane = (long long)v.Xp * v.Yp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % v.nx);
        const long long t = i / v.nx;
        const int y = (int)(t % v.ny);
        const int z = (int)(t / v.ny);
        store_images(dst, v, x, y, z * plane, src[i]);
    }
}

template <typename WT>
__global__ void k_weights_f32(LatticeView v, float* __restrict__ dst) {
    const WT* W = static_cast<const WT*>(v.w);
    const long long N = (long long)v.nx * v.ny * v.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % v.nx);
        const long long t = i / v.nx;
        const int y = (int)(t % v.ny);
        const int z = (int)(t / v.ny);
        const long long p = ((long long)z * v.Yp + y + v.G) * v.Xp + x + v.G;
        for (int k = 0; k < 6; ++k) dst[k * N + i] = ldw<WT>(W + k * v.Np + p);
    }
}

// max_x |a - b| over interior sites (non-negative floats order like their bits).
__global__ void k_maxdiff(const float* __restrict__ a, const float* __restrict__ b, LatticeView v,
                          unsigned int* out) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % v.nx);
        const long long t = i / v.nx;
        const int y = (int)(t % v.ny);
        const int z = (int)(t / v.ny);
        const long long p = ((long long)z * v.Yp + y + v.G) * v.Xp + x + v.G;
        m = fmaxf(m, fabsf(a[p] - b[p]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    const long long cap = (long long)device_props().sm_count * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_pack(const LatticeView& v, int wdtype, const double* F, const double* omega,
                        const uint8_t* solid, double alpha, const double* alpha_links, double dt, double kT,
                        const ResFaces& rf, cudaStream_t st, int z0, int z1) {
    if (z1 < 0) z1 = v.nz;
    const long long plane = (long long)v.Xp * v.Yp;
    const long long p0 = z0 * plane, p1 = z1 * plane;
    if (p1 <= p0) return cudaSuccess;
    const int B = 256;
    const long long g = (p1 - p0 + B - 1) / B;
    if (wdtype == LPC_WEIGHTS_BF16)
        k_pack<__nv_bfloat16><<<(unsigned)g, B, 0, st>>>(v, F, omega, solid, alpha, alpha_links, dt, kT, rf, p0, p1);
    else
        k_pack<float><<<(unsigned)g, B, 0, st>>>(v, F, omega, solid, alpha, alpha_links, dt, kT, rf, p0, p1);
    return cudaGetLastError();
}

namespace {

// The value checks of create on the device copies (bit 0: F not finite on a
// pore site, 1: omega not finite, 2: rho0 not finite on a pore site, 3: a
// link factor outside [0, 1]), or-ed into *bits.
__global__ void k_check_inputs(const double* __restrict__ F, const double* __restrict__ omega,
                               const uint8_t* __restrict__ solid, const double* __restrict__ rho0,
                               const double* __restrict__ links, long long N, unsigned int* bits) {
    unsigned int b = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const bool pore = solid[i] == 0;
        if (pore && !isfinite(F[i])) b |= 1u;
        if (!isfinite(omega[i])) b |= 2u;
        if (rho0 && pore && !isfinite(rho0[i])) b |= 4u;
        if (links)
            for (int a = 0; a < 3; ++a) {
                const double l = links[a * N + i];
                if (!(l >= 0.0 && l <= 1.0)) b |= 8u;
            }
    }
    b = __reduce_or_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && b) atomicOr(bits, b);
}

}  // namespace

cudaError_t launch_check_inputs(const double* F, const double* omega, const uint8_t* solid, const double* rho0,
                                const double* links, long long N, unsigned int* bits, cudaStream_t st) {
    const int B = 256;
    k_check_inputs<<<grid_for(N, B), B, 0, st>>>(F, omega, solid, rho0, links, N, bits);
    return cudaGetLastError();
}

cudaError_t launch_reservoir_ghosts(const LatticeView& v, const ResFaces& rf, cudaStream_t st) {
    if (!rf.any()) return cudaSuccess;
    const int B = 256;
    const long long g = (v.Np + B - 1) / B;
    k_reservoir_ghosts<<<(unsigned)g, B, 0, st>>>(v, rf);
    return cudaGetLastError();
}

namespace {

// Gather form of the static data, read from the padded hop-weight planes:
// win_k(x) = w_k(x - e_k) for the source of each of the six incoming hops
// (plane k at the neighbour the kernels' gather reads: x-1, x+1, y-1, y+1,
// z-1, z+1 for k = 0..5; ghosts hold the periodic images, zero behind
// walls; z wraps, the hop across a z wall being zero), the stay weight with
// the same FP32 sum as the step kernels, R, and the out-weight pair of every
// MSD axis.  With gdx the x pairs are not stored: the x out-weights of a site
// are the in-weights of its x neighbours, which the kernel holds, except at
// the two ends of a 64-column tile, whose values gdx keeps
// ([nz][tiles_x][nyp][2], nyp = ny rounded up to 8 so that rows are 16-byte
// multiples: w_-x of the tile's first column, w_+x of its last site).
// Positions x >= nx of the unpadded pitch get zeros.
template <typename WT>
__global__ void k_gather_pack(LatticeView v, WT* __restrict__ win, float* __restrict__ gs,
                              float2* __restrict__ gR, WT* __restrict__ gdm, WT* __restrict__ gdx) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.Ns) return;
    const int x = (int)(g % v.Xs);
    const long long t = g / v.Xs;
    const int y = (int)(t % v.ny);
    const int z = (int)(t / v.ny);
    const WT* W = static_cast<const WT*>(v.w);
    if (x >= v.nx) {
        for (int k = 0; k < 6; ++k) win[k * v.Ns + g] = round_weight<WT>(0.0);
        gs[g] = 0.0f;
        gR[g] = make_float2(0.0f, 0.0f);
        for (int a = 0; a < 3; ++a)
            if (gdm && (v.msd_axes >> a & 1)) {
                gdm[2 * (a * v.Ns + g)] = round_weight<WT>(0.0);
                gdm[2 * (a * v.Ns + g) + 1] = round_weight<WT>(0.0);
            }
        return;
    }
    const long long zplane = (long long)v.Xp * v.Yp;
    const long long p = (long long)z * zplane + (long long)(y + v.G) * v.Xp + (x + v.G);
    const long long pzm = p + (long long)((z == 0 ? v.nz - 1 : z - 1) - z) * zplane;
    const long long pzp = p + (long long)((z == v.nz - 1 ? 0 : z + 1) - z) * zplane;
    const long long src[6] = {p - 1, p + 1, p - v.Xp, p + v.Xp, pzm, pzp};
    float wo[6];
    for (int k = 0; k < 6; ++k) {
        win[k * v.Ns + g] = W[k * v.Np + src[k]];
        wo[k] = ldw<WT>(W + k * v.Np + p);
    }
    gs[g] = stay_weight(wo);
    gR[g] = v.R[p];
    for (int a = 0; a < 3; ++a)
        if (gdm && (v.msd_axes >> a & 1) && !(a == 0 && gdx)) {
            // the stored out-weights themselves (exact in their own type)
            gdm[2 * (a * v.Ns + g)] = W[(2 * a) * v.Np + p];
            gdm[2 * (a * v.Ns + g) + 1] = W[(2 * a + 1) * v.Np + p];
        }
    if (gdx && x % 64 == 0) {
        const int tiles_x = (v.nx + 63) / 64;
        const int nyp = (v.ny + 7) / 8 * 8;
        const int xl = min(x + 63, v.nx - 1);      // the tile's last site
        const long long e = 2 * (((long long)z * tiles_x + x / 64) * nyp + y);
        gdx[e] = W[1 * v.Np + p];
        gdx[e + 1] = W[0 * v.Np + p + (xl - x)];
    }
}

}  // namespace

namespace {

// Restart of the propagation phase from the current populations: both
// buffers get rho = the current rho (ghost images included), m = rho, mu = 0.
__global__ void k_restart(LatticeView v, const float* __restrict__ rho_cur, float* rho_other, float2* m0,
                          float2* m1, float* mu00, float* mu01, float* mu02, float* mu10, float* mu11,
                          float* mu12) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.Np) return;
    const float r = rho_cur[p];
    rho_other[p] = r;
    m0[p] = make_float2(r, 0.0f);
    m1[p] = make_float2(r, 0.0f);
    float* mu[6] = {mu00, mu01, mu02, mu10, mu11, mu12};
    for (int i = 0; i < 6; ++i)
        if (mu[i]) mu[i][p] = 0.0f;
}

}  // namespace

cudaError_t launch_restart(const LatticeView& v, cudaStream_t st) {
    const int B = 256;
    const long long g = (v.Np + B - 1) / B;
    // v: input = the current state, output = the other buffer
    k_restart<<<(unsigned)g, B, 0, st>>>(v, v.rho_in, v.rho_out, const_cast<float2*>(v.m_in), v.m_out,
                                          const_cast<float*>(v.mu_in[0]), const_cast<float*>(v.mu_in[1]),
                                          const_cast<float*>(v.mu_in[2]), v.mu_out[0], v.mu_out[1], v.mu_out[2]);
    return cudaGetLastError();
}

namespace {

template <typename WT> __device__ __forceinline__ float wt_to_float(WT w);
template <> __device__ __forceinline__ float wt_to_float<float>(float w) { return w; }
template <> __device__ __forceinline__ float wt_to_float<__nv_bfloat16>(__nv_bfloat16 w) { return __bfloat162float(w); }

// Link form of the static data of a lattice with one jump factor: for every
// site y and axis a the link to y + e_a as one signed value L (0: closed;
// L > 0: the hop y -> y + e_a weighs L and the hop back A; L < 0: the hop
// y -> y + e_a weighs A and the hop back -L), A = alpha/6 rounded like the
// hop weights (the weight of a downhill or level Metropolis move, Eq. 1;
// reservoir links follow the same rule).  Read from the padded out-weights
// (ghost images, walls and reservoir ghosts included), so the weights the
// kernel rebuilds are the stored ones.  Rows of pitch Xs, ny + 1 rows per
// plane: row 0 holds the link that enters row 0 from below (from the image
// of row ny - 1 on a periodic y axis, from the ghost row otherwise: a
// reservoir's link, or closed at a wall).  X0 [nz][ny] holds the link that
// enters column 0 from the left in the same way.  R is copied to rows of
// pitch Xs.  `bad` is set when a link does not fit the form (an open link
// whose small hop rounded to zero, or no hop equal to A); `a_out` receives A
// as a float.
__device__ __forceinline__ float link_value(float wf, float wb, float A, unsigned int* bad) {
    if (wf == 0.0f && wb == 0.0f) return 0.0f;
    if (wb == A && wf > 0.0f) return wf;
    if (wf == A && wb > 0.0f) return -wb;
    atomicOr(bad, 1u);
    return 0.0f;
}

template <typename WT>
__global__ void k_link_pack(LatticeView v, WT* __restrict__ L, WT* __restrict__ X0, float2* __restrict__ Rl,
                            double alpha, unsigned int* __restrict__ bad, float* __restrict__ a_out) {
    const WT* W = static_cast<const WT*>(v.w);
    const float A = wt_to_float<WT>(round_weight<WT>(alpha / 6.0 * 1.0));
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (gid == 0) *a_out = A;
    const long long zp = (long long)v.Xp * v.Yp;
    const long long total = 3LL * v.nz * v.ny1 * v.Xs;
    for (long long g = gid; g < total; g += stride) {
        const int x = (int)(g % v.Xs);
        const long long t = g / v.Xs;
        const int row = (int)(t % v.ny1);
        const long long t2 = t / v.ny1;
        const int z = (int)(t2 % v.nz);
        const int a = (int)(t2 / v.nz);
        int y = row - 1;
        if (row == 0 && v.per_y) y = v.ny - 1;
        float val = 0.0f;
        // y = -1: the ghost row below row 0 (its weights: 0 at a wall, a
        // reservoir's at a reservoir face); only y links start there
        if (x < v.nx && (y >= 0 || a == 1)) {
            const long long p = z * zp + (long long)(y + v.G) * v.Xp + (x + v.G);
            const long long pn = a == 0 ? p + 1
                                 : a == 1 ? p + v.Xp
                                          : (long long)(z + 1 == v.nz ? 0 : z + 1) * zp + (p - z * zp);
            const float wf = ldw<WT>(W + (long long)(2 * a) * v.Np + p);
            const float wb = ldw<WT>(W + (long long)(2 * a + 1) * v.Np + pn);
            val = link_value(wf, wb, A, bad);
        }
        L[g] = round_weight<WT>((double)val);
    }
    // links entering column 0 from the left: from the ghost column (the image
    // of column nx - 1 on a periodic x axis, a reservoir ghost, or a wall)
    const long long nx0 = (long long)v.nz * v.ny;
    for (long long g = gid; g < nx0; g += stride) {
        const int y = (int)(g % v.ny);
        const int z = (int)(g / v.ny);
        const long long p = z * zp + (long long)(y + v.G) * v.Xp + (v.G - 1);
        const float wf = ldw<WT>(W + p);
        const float wb = ldw<WT>(W + v.Np + p + 1);
        X0[g] = round_weight<WT>((double)link_value(wf, wb, A, bad));
    }
    const long long nr = (long long)v.nz * v.ny * v.Xs;
    for (long long g = gid; g < nr; g += stride) {
        const int x = (int)(g % v.Xs);
        const long long t = g / v.Xs;
        const int y = (int)(t % v.ny);
        const int z = (int)(t / v.ny);
        Rl[g] = x < v.nx ? v.R[z * zp + (long long)(y + v.G) * v.Xp + (x + v.G)] : make_float2(0.0f, 0.0f);
    }
}

}  // namespace

cudaError_t launch_link_pack(const LatticeView& v, int wdtype, void* L, void* X0, float2* Rl, double alpha,
                             unsigned int* bad, float* a_out, cudaStream_t st) {
    const long long total = 3LL * v.nz * v.ny1 * v.Xs;
    const int g = grid_for(total, 256);
    if (wdtype == LPC_WEIGHTS_BF16)
        k_link_pack<__nv_bfloat16><<<g, 256, 0, st>>>(v, static_cast<__nv_bfloat16*>(L),
                                                      static_cast<__nv_bfloat16*>(X0), Rl, alpha, bad, a_out);
    else
        k_link_pack<float><<<g, 256, 0, st>>>(v, static_cast<float*>(L), static_cast<float*>(X0), Rl, alpha, bad,
                                              a_out);
    return cudaGetLastError();
}

// Pitch of the gather-form arrays: rows start on 256-byte boundaries.
int gather_pitch(int nx) { return (nx + 63) / 64 * 64; }

cudaError_t launch_gather_pack(const LatticeView& v, int wdtype, void* win, float* s, float2* R, void* dm, void* dx,
                               cudaStream_t st) {
    const int B = 256;
    const long long g = (v.Ns + B - 1) / B;
    if (wdtype == LPC_WEIGHTS_BF16)
        k_gather_pack<__nv_bfloat16><<<(unsigned)g, B, 0, st>>>(v, static_cast<__nv_bfloat16*>(win), s, R,
                                                                static_cast<__nv_bfloat16*>(dm),
                                                                static_cast<__nv_bfloat16*>(dx));
    else
        k_gather_pack<float><<<(unsigned)g, B, 0, st>>>(v, static_cast<float*>(win), s, R, static_cast<float*>(dm),
                                                        static_cast<float*>(dx));
    return cudaGetLastError();
}

cudaError_t launch_init_state(const LatticeView& v, const double* rho0_dev, int init_mode,
                              const double* F, const uint8_t* solid, double kT, double* scratch,
                              cudaStream_t st) {
    // the normalisation of Eq. 2 runs over the own planes [zlo, zhi) (halo
    // planes of z reservoirs hold reservoir sites)
    const long long plane = (long long)v.nx * v.ny;
    const long long N = plane * (v.zhi - v.zlo);
    const double* zsum = nullptr;
    if (!rho0_dev && init_mode == LPC_INIT_BOLTZMANN) {
        const int nb = 256;
        k_boltz_partial<<<nb, 256, 0, st>>>(F + v.zlo * plane, solid + v.zlo * plane, N, kT, scratch);
        k_boltz_final<<<1, 32, 0, st>>>(scratch, nb);
        zsum = scratch + 2 * nb;
    }
    const int B = 256;
    const long long g = (v.Np + B - 1) / B;
    k_init<<<(unsigned)g, B, 0, st>>>(v, rho0_dev, init_mode, F, solid, kT, zsum);
    return cudaGetLastError();
}

cudaError_t launch_sum_state(const LatticeView& v, cudaStream_t st) {
    const long long rows = (long long)v.ny * v.nz * ((v.nx + 31) / 32);
    long long g = (rows + 7) / 8;
    const long long cap = (long long)device_props().sm_count * 8;
    if (g > cap) g = cap;
    k_sum_state<<<(unsigned)g, dim3(32, 8), 0, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_unpad(const void* src, int elem_bytes, const LatticeView& v, void* dst_dev,
                         cudaStream_t st) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    const int g = grid_for(N, 256);
    if (elem_bytes == 8)
        k_unpad<float2><<<g, 256, 0, st>>>(static_cast<const float2*>(src), v, static_cast<float2*>(dst_dev));
    else
        k_unpad<float><<<g, 256, 0, st>>>(static_cast<const float*>(src), v, static_cast<float*>(dst_dev));
    return cudaGetLastError();
}

cudaError_t launch_pad(const void* src_dev, int elem_bytes, const LatticeView& v, void* dst,
                       cudaStream_t st) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    const int g = grid_for(N, 256);
    if (elem_bytes == 8)
        k_pad<float2><<<g, 256, 0, st>>>(static_cast<const float2*>(src_dev), v, static_cast<float2*>(dst));
    else
        k_pad<float><<<g, 256, 0, st>>>(static_cast<const float*>(src_dev), v, static_cast<float*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_weights_f32(const LatticeView& v, int wdtype, float* dst_dev, cudaStream_t st) {
    const long long N = (long long)v.nx * v.ny * v.nz;
    const int g = grid_for(N, 256);
    if (wdtype == LPC_WEIGHTS_BF16) k_weights_f32<__nv_bfloat16><<<g, 256, 0, st>>>(v, dst_dev);
    else k_weights_f32<float><<<g, 256, 0, st>>>(v, dst_dev);
    return cudaGetLastError();
}

cudaError_t launch_maxdiff(const float* a, const float* b, const LatticeView& v, double* out2,
                           cudaStream_t st) {
    unsigned int* u = reinterpret_cast<unsigned int*>(out2);
    cudaError_t e = cudaMemsetAsync(u, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const long long N = (long long)v.nx * v.ny * v.nz;
    k_maxdiff<<<grid_for(N, 256), 256, 0, st>>>(a, b, v, u);
    return cudaGetLastError();
}

}  // namespace lpc
