// One time step per launch fed by TMA with warp specialisation (the TB
// schedule at block depth 1).
//
// A CTA owns a core tile of 32 x TY (x, y) columns (TY = NC consumer warps x
// RPW rows per warp) and walks z-chunks of it.  A producer warp streams,
// plane by plane, a W x (TY + 2) box (W = 32 + 2G rounded up to 16 bytes: the
// core plus the G-wide ghost bands in x; one halo row above and below) of the
// state (rho, m, mu), the six hop-weight planes (one 4-D box) and R into a
// ring of S shared-memory slots with cp.async.bulk.tensor; each slot has a
// "full" mbarrier (TMA transaction bytes) and an "empty" mbarrier (one
// arrival per consumer warp).  Consumer warps wait for the plane above,
// update their rows from shared memory (all six neighbours are in the ring:
// x and y in the slot of the plane, z above from the ring and z below from
// registers) and release the plane.  No block-wide barrier is needed inside the loop,
// and the ring keeps up to S planes of HBM reads in flight without holding
// registers.  Tile shapes 32 x 32, 32 x 16 (one CTA per SM) or 32 x 8 (two
// per SM): the largest whose ring holds six planes.  Ring positions advance as
// cursors (no divisions in the loop).  Per-site arithmetic is the shared
// site function, so states are bit-identical to the other kernels.
//
// Every wait is bounded (clock64 budget); on expiry the kernel records
// LPC_ERR_TIMEOUT in the lattice's error word, waits (bounded) for its
// copies in flight and returns without writing the step's sums.
#include "lpc_internal.cuh"
#include "tma_ptx.cuh"

namespace lpc {

namespace {

template <typename WT> __device__ __forceinline__ float sw(const WT* p);
template <> __device__ __forceinline__ float sw<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float sw<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __uint_as_float(static_cast<unsigned int>(*reinterpret_cast<const unsigned short*>(p)) << 16);
}

constexpr int popc(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

// Position in the slot ring: slot index and the parity of its barrier phase.
struct Cursor {
    int slot;
    unsigned int ph;
    __device__ __forceinline__ void next(int S) {
        if (++slot == S) { slot = 0; ph ^= 1u; }
    }
};

}  // namespace

struct T1Geom {
    int W, S, cz;
    int tiles_x, tiles_y, n_items;
    int slot_bytes, tx_bytes;
    unsigned int* err;
};

namespace {

// slot layout (each part starts on a 128-byte boundary, as TMA requires):
//   rho [H][W] f32 | m [H][W] f32x2 | mu_n [H][W] f32 | w [6][H][W] WT |
//   R [H][W] f32x2
struct T1Slot {
    int m, mu[3], w, R, bytes;
};
__host__ __device__ inline int up128(int n) { return (n + 127) / 128 * 128; }
__host__ __device__ inline T1Slot t1_slot(int W, int H, int nmsd, int wb) {
    T1Slot L;
    const int HW = H * W;
    int off = up128(HW * 4);
    L.m = off;
    off += up128(HW * 8);
    for (int n = 0; n < 3; ++n) {
        L.mu[n] = off;
        if (n < nmsd) off += up128(HW * 4);
    }
    L.w = off;
    off += up128(HW * 6 * wb);
    L.R = off;
    off += up128(HW * 8);
    L.bytes = off;
    return L;
}

template <typename WT, int MSD, int NC, int RPW>
__global__ void __launch_bounds__((NC + 1) * 32, NC > 8 ? 1 : 2)
k_step_tma1(const __grid_constant__ TBMaps maps, LatticeView v, T1Geom g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (sa(smem_raw) & 127u)) & 127u);
    constexpr int NMSD = popc(MSD);
    constexpr int TY = NC * RPW;              // core rows
    constexpr int H = TY + 2;                 // box rows
    const int W = g.W, S = g.S, HW = H * W;
    const T1Slot SL = t1_slot(W, H, NMSD, (int)sizeof(WT));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * g.slot_bytes);
    uint64_t* empty = full + S;
    double* red = reinterpret_cast<double*>(empty + S);          // [NC+1][kNumSums]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(red + (NC + 1) * kNumSums);
    volatile unsigned int* issued = reinterpret_cast<volatile unsigned int*>(abort_flag + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = v.G;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC);
        }
        *abort_flag = 0;
        *issued = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < (NC + 1) * kNumSums; i += (NC + 1) * 32) red[i] = 0.0;
    __syncthreads();

    int axis_of[3] = {0, 0, 0};
    {
        int n = 0;
        for (int a = 0; a < 3; ++a)
            if (MSD >> a & 1) axis_of[n++] = a;
    }
    const long long zplane = (long long)v.Xp * v.Yp;

    if (warp == NC) {
        // ---------------- producer warp: one elected lane issues the copies
        if (lane == 0) {
            bool ok = true;
            Cursor c{0, 0u};
            unsigned int n_loads = 0;
            for (int item = blockIdx.x; item < g.n_items && ok; item += gridDim.x) {
                const int tx = item % g.tiles_x;
                const int rest = item / g.tiles_x;
                const int ty = rest % g.tiles_y;
                const int zc = rest / g.tiles_y;
                const int bx = tx * 32, by = ty * TY - 1 + G;   // box origin (padded)
                const int z0 = zc * g.cz;
                const int CZ = min(g.cz, v.nz - z0);
                int z = z0 - 1 < 0 ? v.nz - 1 : z0 - 1;
                for (int i = 0; i < CZ + 2; ++i) {
                    // the slot's previous plane must be released by every consumer
                    if (n_loads >= (unsigned)S) ok = mbar_wait_bounded(&empty[c.slot], c.ph ^ 1u);
                    if (!ok || *abort_flag) { ok = false; break; }
                    unsigned char* st = smem + (size_t)c.slot * g.slot_bytes;
                    uint64_t* fb = &full[c.slot];
                    fence_proxy_async();
                    mbar_expect_tx(fb, (uint32_t)g.tx_bytes);
                    tma3(st, &maps.rho, fb, bx, by, z);
                    tma3(st + SL.m, &maps.m, fb, 2 * bx, by, z);
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) tma3(st + SL.mu[n], &maps.mu[n], fb, bx, by, z);
                    tma4(st + SL.w, &maps.w, fb, bx, by, z, 0);
                    tma3(st + SL.R, &maps.R, fb, 2 * bx, by, z);
                    *issued = ++n_loads;
                    c.next(S);
                    if (++z == v.nz) z = 0;
                }
            }
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---------------- consumer warps: rows warp + 1 + j*NC of the box
        // A thread keeps its own column of the plane below in registers (the
        // only part of that plane the update reads), so it holds just two
        // slots (this plane and the one above) and releases a plane as soon
        // as it has been the centre.
        float part[kNumSums] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool ok = true;
        Cursor wait_c{0, 0u};          // next load to wait for
        for (int item = blockIdx.x; item < g.n_items && ok; item += gridDim.x) {
            const int tx = item % g.tiles_x;
            const int rest = item / g.tiles_x;
            const int ty = rest % g.tiles_y;
            const int zc = rest / g.tiles_y;
            const int x = tx * 32 + lane;
            const int z0 = zc * g.cz;
            const int CZ = min(g.cz, v.nz - z0);
            // per-row facts of this item
            bool site[RPW], inner[RPW];
            int y[RPW], o[RPW];
            long long col[RPW];
#pragma unroll
            for (int j = 0; j < RPW; ++j) {
                y[j] = ty * TY + warp + j * NC;
                site[j] = x < v.nx && y[j] < v.ny;
                inner[j] = x >= G && x < v.nx - G && y[j] >= G && y[j] < v.ny - G;
                col[j] = (long long)(y[j] + G) * v.Xp + (x + G) + (long long)z0 * zplane;
                o[j] = (warp + 1 + j * NC) * W + G + lane;
            }
            // plane 0 of the item: keep this thread's column as "below"
            float br[RPW], bw4[RPW], bmu[RPW][3];
            float2 bm[RPW];
            ok = mbar_wait_bounded(&full[wait_c.slot], wait_c.ph);
            if (!ok) break;
            {
                const unsigned char* s0 = smem + (size_t)wait_c.slot * g.slot_bytes;
#pragma unroll
                for (int j = 0; j < RPW; ++j) {
                    br[j] = reinterpret_cast<const float*>(s0)[o[j]];
                    bm[j] = reinterpret_cast<const float2*>(s0 + SL.m)[o[j]];
                    bw4[j] = sw<WT>(reinterpret_cast<const WT*>(s0 + SL.w) + 4 * HW + o[j]);
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) bmu[j][n] = reinterpret_cast<const float*>(s0 + SL.mu[n])[o[j]];
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[wait_c.slot]);
                wait_c.next(S);
            }
            // plane 1: the first centre
            ok = mbar_wait_bounded(&full[wait_c.slot], wait_c.ph);
            int center = wait_c.slot;
            wait_c.next(S);
            for (int q = 0; q < CZ && ok; ++q) {
                const int above = wait_c.slot;
                ok = mbar_wait_bounded(&full[above], wait_c.ph);
                wait_c.next(S);
                if (!ok || *abort_flag) { ok = false; break; }
                const unsigned char* sc = smem + (size_t)center * g.slot_bytes;
                const unsigned char* sa_ = smem + (size_t)above * g.slot_bytes;
                const float* rc = reinterpret_cast<const float*>(sc);
                const float* ra = reinterpret_cast<const float*>(sa_);
                const float2* mc = reinterpret_cast<const float2*>(sc + SL.m);
                const float2* ma = reinterpret_cast<const float2*>(sa_ + SL.m);
                const WT* wc = reinterpret_cast<const WT*>(sc + SL.w);
                const WT* wa = reinterpret_cast<const WT*>(sa_ + SL.w);
                const float2* Rc = reinterpret_cast<const float2*>(sc + SL.R);
#pragma unroll
                for (int j = 0; j < RPW; ++j) {
                    const int oj = o[j];
                    SiteIn qi;
                    float wo[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) wo[k] = sw<WT>(wc + k * HW + oj);
                    qi.rc = rc[oj];
                    qi.mc = mc[oj];
                    float muc[3];
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) muc[n] = reinterpret_cast<const float*>(sc + SL.mu[n])[oj];
                    if (site[j]) {
                        qi.r[0] = rc[oj - 1];  qi.m[0] = mc[oj - 1];  qi.win[0] = sw<WT>(wc + 0 * HW + oj - 1);
                        qi.r[1] = rc[oj + 1];  qi.m[1] = mc[oj + 1];  qi.win[1] = sw<WT>(wc + 1 * HW + oj + 1);
                        qi.r[2] = rc[oj - W];  qi.m[2] = mc[oj - W];  qi.win[2] = sw<WT>(wc + 2 * HW + oj - W);
                        qi.r[3] = rc[oj + W];  qi.m[3] = mc[oj + W];  qi.win[3] = sw<WT>(wc + 3 * HW + oj + W);
                        qi.r[4] = br[j];       qi.m[4] = bm[j];       qi.win[4] = bw4[j];
                        qi.r[5] = ra[oj];      qi.m[5] = ma[oj];      qi.win[5] = sw<WT>(wa + 5 * HW + oj);
#pragma unroll
                        for (int k = 0; k < 6; ++k) qi.wout[k] = wo[k];
                        qi.R = Rc[oj];
                        const float s_ = stay_weight(wo);
                        float ro;
                        float2 mo;
                        site_rho_m(qi, s_, ro, mo);
                        const long long zoff = (long long)(z0 + q) * zplane;
                        if (inner[j]) {
                            const long long p = col[j] + (long long)q * zplane;
                            v.rho_out[p] = ro;
                            v.m_out[p] = mo;
                        } else {
                            store_images(v.rho_out, v, x, y[j], zoff, ro);
                            store_images(v.m_out, v, x, y[j], zoff, mo);
                        }
                        part[0] += mo.x;
                        part[1] += mo.y;
                        part[2] += ro;
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) {
                            const int a = axis_of[n];
                            const float* uc = reinterpret_cast<const float*>(sc + SL.mu[n]);
                            const float* ua = reinterpret_cast<const float*>(sa_ + SL.mu[n]);
                            const float nb[6] = {uc[oj - 1], uc[oj + 1], uc[oj - W], uc[oj + W], bmu[j][n], ua[oj]};
                            const float muo = site_mu(qi.win, qi.r, nb, s_, muc[n], a);
                            store_images(v.mu_out[a], v, x, y[j], zoff, muo);
                            part[3 + a] += site_dmsd(wo, muc[n], qi.rc, a);
                        }
                    }
                    // this plane is the next one's "below"
                    br[j] = qi.rc;
                    bm[j] = qi.mc;
                    bw4[j] = wo[4];
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) bmu[j][n] = muc[n];
                }
                // the centre plane is no longer needed by this warp
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[center]);
                center = above;
            }
            if (ok) {
                // release the last plane of the item (loaded as the final "above")
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[center]);
            }
        }
        if (!ok) *abort_flag = 1;
        // per-warp FP64 sums (one butterfly per quantity for the whole launch)
#pragma unroll
        for (int qq = 0; qq < kNumSums; ++qq) {
            if (qq >= 3 && !(MSD >> (qq - 3) & 1)) continue;
            const float t = warp_sum_f32(part[qq]);
            if (lane == 0) red[warp * kNumSums + qq] = (double)t;
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            atomicExch(g.err, (unsigned int)LPC_ERR_TIMEOUT);
            // wait (bounded) until the copies of the last S issued loads landed
            const unsigned int n_issued = *issued;
            for (unsigned int l = n_issued > (unsigned)S ? n_issued - S : 0; l < n_issued; ++l)
                mbar_wait_bounded(&full[l % S], (l / S) & 1u);
        }
        __syncthreads();
        return;
    }
    block_finish_smem<NC + 1>(v, 1, red);
}

template <typename WT, int MSD, int NC, int RPW>
void* t1_fn() { return reinterpret_cast<void*>(&k_step_tma1<WT, MSD, NC, RPW>); }

template <int NC, int RPW>
void* t1_kernel_shape(int wdtype, int msd) {
    static void* tab[2][8] = {
        {t1_fn<float, 0, NC, RPW>(), t1_fn<float, 1, NC, RPW>(), t1_fn<float, 2, NC, RPW>(),
         t1_fn<float, 3, NC, RPW>(), t1_fn<float, 4, NC, RPW>(), t1_fn<float, 5, NC, RPW>(),
         t1_fn<float, 6, NC, RPW>(), t1_fn<float, 7, NC, RPW>()},
        {t1_fn<__nv_bfloat16, 0, NC, RPW>(), t1_fn<__nv_bfloat16, 1, NC, RPW>(),
         t1_fn<__nv_bfloat16, 2, NC, RPW>(), t1_fn<__nv_bfloat16, 3, NC, RPW>(),
         t1_fn<__nv_bfloat16, 4, NC, RPW>(), t1_fn<__nv_bfloat16, 5, NC, RPW>(),
         t1_fn<__nv_bfloat16, 6, NC, RPW>(), t1_fn<__nv_bfloat16, 7, NC, RPW>()}};
    return tab[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
}

// Tile shapes (consumer warps x rows per warp): 16 x 2 (32 x 32 core) or
// 16 x 1 (32 x 16 core) with one CTA per SM, and 8 x 1 (32 x 8 core) with two
// CTAs per SM.  The largest shape whose ring holds at least kMinSlots planes
// is used.
constexpr int kMinSlots = 6;

struct T1Choice {
    int shape;                 // 0: 16 x 2, 1: 16 x 1, 2: 8 x 1
    int W, H, S, slot_bytes, smem;
};

}  // namespace

// Box width of the depth-1 kernel: the 32 core columns plus G on each side,
// rounded up to 16 bytes of the narrowest element (4 FP32, 8 BF16 weights).
int t1_box_width(int G, int wdtype) {
    const int a = wdtype == LPC_WEIGHTS_BF16 ? 8 : 4;
    return (32 + 2 * G + a - 1) / a * a;
}

static T1Choice t1_choose(const LatticeView& v, int wdtype) {
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    const int nmsd = popc(v.msd_axes);
    T1Choice c;
    c.W = t1_box_width(v.G, wdtype);
    const int fixed = 128 + 2048 + 16;
    const int rows[3] = {32, 16, 8};
    const int per_sm[3] = {1, 1, 2};
    for (int shape = 0; shape < 3; ++shape) {
        const int H = rows[shape] + 2;
        const int sb = t1_slot(c.W, H, nmsd, wb).bytes;
        int S = (device_props().max_smem_optin / per_sm[shape] - fixed) / (sb + 16);
        if (S > 8) S = 8;
        const bool last = shape == 2;
        if ((S >= kMinSlots && v.ny > rows[shape] / 2) || last) {
            if (S < 4) S = 4;
            c.shape = shape;
            c.H = H;
            c.S = S;
            c.slot_bytes = sb;
            c.smem = fixed + S * (sb + 16);
            return c;
        }
    }
    return c;
}

int t1_box_rows(const LatticeView& v, int wdtype) { return t1_choose(v, wdtype).H; }

static void* t1_kernel(const T1Choice& c, int wdtype, int msd) {
    if (c.shape == 0) return t1_kernel_shape<16, 2>(wdtype, msd);
    if (c.shape == 1) return t1_kernel_shape<16, 1>(wdtype, msd);
    return t1_kernel_shape<8, 1>(wdtype, msd);
}

cudaError_t t1_prepare(int wdtype, int msd) {
    static bool done[2][8] = {};
    bool& d = done[wdtype == LPC_WEIGHTS_BF16][msd & 7];
    if (d) return cudaSuccess;
    void* fns[3] = {t1_kernel_shape<16, 2>(wdtype, msd), t1_kernel_shape<16, 1>(wdtype, msd),
                    t1_kernel_shape<8, 1>(wdtype, msd)};
    const int limit[3] = {device_props().max_smem_optin, device_props().max_smem_optin,
                          device_props().max_smem_optin / 2};
    for (int i = 0; i < 3; ++i) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fns[i]);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 limit[i] - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    d = true;
    return cudaSuccess;
}

cudaError_t launch_tma1(const LatticeView& v, int wdtype, const TBMaps& maps, unsigned int* err,
                        cudaStream_t st) {
    const T1Choice c = t1_choose(v, wdtype);
    const int nmsd = popc(v.msd_axes);
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    const int NC = c.shape == 2 ? 8 : 16;
    const int TY = c.shape == 0 ? 32 : (c.shape == 1 ? 16 : 8);
    T1Geom g;
    g.W = c.W;
    g.S = c.S;
    g.slot_bytes = c.slot_bytes;
    g.tx_bytes = c.H * c.W * (4 + 8 + 4 * nmsd + 6 * wb + 8);   // the boxes (padding not written)
    g.tiles_x = (v.nx + 31) / 32;
    g.tiles_y = (v.ny + TY - 1) / TY;
    const long long xy = (long long)g.tiles_x * g.tiles_y;
    const int ctas = device_props().sm_count * (c.shape == 2 ? 2 : 1);
    const long long nchunks = (4LL * ctas + xy - 1) / xy;     // ~4 items per CTA
    int cz = (int)((v.nz + nchunks - 1) / nchunks);
    if (cz < 16) cz = 16;
    if (cz > v.nz) cz = v.nz;
    g.cz = cz;
    g.n_items = (int)(xy * ((v.nz + cz - 1) / cz));
    g.err = err;
    cudaError_t e = t1_prepare(wdtype, v.msd_axes);
    if (e != cudaSuccess) return e;
    int grid = ctas;
    if (grid > g.n_items) grid = g.n_items;
    LatticeView vv = v;
    TBMaps mm = maps;
    void* args[] = {&mm, &vv, &g};
    return cudaLaunchKernel(t1_kernel(c, wdtype, v.msd_axes), dim3(grid), dim3((NC + 1) * 32), args,
                            (size_t)c.smem, st);
}

}  // namespace lpc
