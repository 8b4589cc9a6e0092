// One time step per launch (the "step1" schedule).
//
// A block of 32 x 8 threads owns a 32 x 8 column of (x, y) sites and walks a
// chunk of z planes; each thread keeps the state and the hop weights of the
// planes below, at and above its site in registers, so only the four in-plane
// neighbours are re-read (from L1/L2).  Blocks loop over (x-tile, y-tile,
// z-chunk) work items with a grid of SM count x resident blocks.  Every warp
// reduces its 32-site row of each plane in FP32 (fixed butterfly) and
// accumulates the row sums in FP64; blocks then combine in FP64 and the last
// block writes the step's M, P and dMSD into the device history.
#include "lpc_internal.cuh"

namespace lpc {

namespace {

constexpr int BX = 32, BY = 8, NWARP = BX * BY / 32;

template <typename WT, int MSD>
__global__ void __launch_bounds__(BX * BY, MSD ? 3 : 4)
k_step1(LatticeView v, int cz, int tiles_x, int tiles_y, int n_items) {
    __shared__ double smem[NWARP * kNumSums];
    const WT* W = static_cast<const WT*>(v.w);
    const long long Np = v.Np;
    const long long plane = (long long)v.Xp * v.Yp;
    const int lane = threadIdx.x;
    double acc[1][kNumSums] = {{0, 0, 0, 0, 0, 0}};

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tx = item % tiles_x;
        const int rest = item / tiles_x;
        const int tyi = rest % tiles_y;
        const int zc = rest / tiles_y;
        const int x = tx * BX + lane;
        const int y = tyi * BY + threadIdx.y;
        const int z0 = zc * cz;
        const int z1 = min(z0 + cz, v.nz);
        const bool act = x < v.nx && y < v.ny;
        const long long col = (long long)(y + v.G) * v.Xp + (x + v.G);

        // registers: b = plane below, c = this plane, n = plane above
        float rb = 0.f, rc = 0.f, w4b = 0.f;
        float2 mb = make_float2(0.f, 0.f), mc = mb;
        float mub[3] = {0.f, 0.f, 0.f}, muc[3] = {0.f, 0.f, 0.f};
        float wc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (act) {
            const int zb = z0 == 0 ? v.nz - 1 : z0 - 1;
            const long long ib = zb * plane + col, ic = z0 * plane + col;
            rb = __ldg(v.rho_in + ib);
            mb = __ldg(v.m_in + ib);
            rc = __ldg(v.rho_in + ic);
            mc = __ldg(v.m_in + ic);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (MSD >> a & 1) { mub[a] = __ldg(v.mu_in[a] + ib); muc[a] = __ldg(v.mu_in[a] + ic); }
            w4b = ldw<WT>(W + 4 * Np + ib);
#pragma unroll
            for (int k = 0; k < 6; ++k) wc[k] = ldw<WT>(W + k * Np + ic);
        }
        for (int z = z0; z < z1; ++z) {
            const int zn = z + 1 == v.nz ? 0 : z + 1;
            const long long ic = z * plane + col, in = zn * plane + col;
            float vals[kNumSums] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float rn = 0.f;
            float2 mn = make_float2(0.f, 0.f);
            float mun[3] = {0.f, 0.f, 0.f};
            float wn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (act) {
                rn = __ldg(v.rho_in + in);
                mn = __ldg(v.m_in + in);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (MSD >> a & 1) mun[a] = __ldg(v.mu_in[a] + in);
#pragma unroll
                for (int k = 0; k < 6; ++k) wn[k] = ldw<WT>(W + k * Np + in);

                // sources of the hops into this site: k = +x from x-1, -x from
                // x+1, +y from y-1, -y from y+1, +z from below, -z from above
                const long long src[4] = {ic - 1, ic + 1, ic - v.Xp, ic + v.Xp};
                SiteIn q;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    q.win[k] = ldw<WT>(W + k * Np + src[k]);
                    q.r[k] = __ldg(v.rho_in + src[k]);
                    q.m[k] = __ldg(v.m_in + src[k]);
                }
                q.win[4] = w4b; q.r[4] = rb; q.m[4] = mb;
                q.win[5] = wn[5]; q.r[5] = rn; q.m[5] = mn;
#pragma unroll
                for (int k = 0; k < 6; ++k) q.wout[k] = wc[k];
                q.rc = rc;
                q.mc = mc;
                q.R = __ldg(v.R + ic);
                const float s = stay_weight(wc);
                float ro;
                float2 mo;
                site_rho_m(q, s, ro, mo);
                const long long zoff = z * plane;
                store_images(v.rho_out, v, x, y, zoff, ro);
                store_images(v.m_out, v, x, y, zoff, mo);
                vals[0] = mo.x;
                vals[1] = mo.y;
                vals[2] = ro;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (!(MSD >> a & 1)) continue;
                    float nbm[6];
#pragma unroll
                    for (int k = 0; k < 4; ++k) nbm[k] = __ldg(v.mu_in[a] + src[k]);
                    nbm[4] = mub[a];
                    nbm[5] = mun[a];
                    const float mo_a = site_mu(q.win, q.r, nbm, s, muc[a], a);
                    store_images(v.mu_out[a], v, x, y, zoff, mo_a);
                    vals[3 + a] = site_dmsd(wc, muc[a], rc, a);
                }
            }
#pragma unroll
            for (int qq = 0; qq < kNumSums; ++qq) {
                if (qq >= 3 && !(MSD >> (qq - 3) & 1)) continue;
                const float t = warp_sum_f32(vals[qq]);
                if (lane == 0) acc[0][qq] += (double)t;
            }
            rb = rc; mb = mc; rc = rn; mc = mn; w4b = wc[4];
#pragma unroll
            for (int a = 0; a < 3; ++a) { mub[a] = muc[a]; muc[a] = mun[a]; }
#pragma unroll
            for (int k = 0; k < 6; ++k) wc[k] = wn[k];
        }
    }
    block_finish<NWARP>(v, acc, 1, smem);
}

template <typename WT, int MSD>
void* step1_fn() { return reinterpret_cast<void*>(&k_step1<WT, MSD>); }

void* step1_kernel(int wdtype, int msd) {
    static void* tab[2][8] = {
        {step1_fn<float, 0>(), step1_fn<float, 1>(), step1_fn<float, 2>(), step1_fn<float, 3>(),
         step1_fn<float, 4>(), step1_fn<float, 5>(), step1_fn<float, 6>(), step1_fn<float, 7>()},
        {step1_fn<__nv_bfloat16, 0>(), step1_fn<__nv_bfloat16, 1>(), step1_fn<__nv_bfloat16, 2>(),
         step1_fn<__nv_bfloat16, 3>(), step1_fn<__nv_bfloat16, 4>(), step1_fn<__nv_bfloat16, 5>(),
         step1_fn<__nv_bfloat16, 6>(), step1_fn<__nv_bfloat16, 7>()}};
    return tab[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
}

struct Step1Shape {
    int cz, tiles_x, tiles_y, n_items, grid;
};

Step1Shape step1_shape(const LatticeView& v, int wdtype) {
    Step1Shape s;
    s.tiles_x = (v.nx + BX - 1) / BX;
    s.tiles_y = (v.ny + BY - 1) / BY;
    static int occ_cache[2][8] = {{0}};
    int& occ = occ_cache[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][v.msd_axes & 7];
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step1_kernel(wdtype, v.msd_axes), BX * BY, 0);
        if (occ < 1) occ = 1;
    }
    const long long resident = (long long)device_props().sm_count * occ;
    // z chunks: enough work items for ~8 waves, chunks of 8..64 planes
    const long long xy = (long long)s.tiles_x * s.tiles_y;
    long long want = resident * 8;
    long long nchunks = (want + xy - 1) / xy;
    int cz = (int)((v.nz + nchunks - 1) / nchunks);
    if (cz > 64) cz = 64;
    if (cz < 8) cz = 8;
    if (cz > v.nz) cz = v.nz;
    s.cz = cz;
    const long long nzc = (v.nz + cz - 1) / cz;
    s.n_items = (int)(xy * nzc);
    s.grid = (int)(resident < s.n_items ? resident : s.n_items);
    return s;
}

}  // namespace

int step1_grid(const LatticeView& v, int wdtype) { return step1_shape(v, wdtype).grid; }

cudaError_t launch_step1(const LatticeView& v, int wdtype, cudaStream_t st) {
    const Step1Shape s = step1_shape(v, wdtype);
    void* fn = step1_kernel(wdtype, v.msd_axes);
    LatticeView vv = v;
    int cz = s.cz, tx = s.tiles_x, ty = s.tiles_y, ni = s.n_items;
    void* args[] = {&vv, &cz, &tx, &ty, &ni};
    return cudaLaunchKernel(fn, dim3(s.grid), dim3(BX, BY), args, 0, st);
}

}  // namespace lpc
