// Temporally blocked step kernel (the "TB" schedule): K time steps per launch.
//
// A CTA owns a core tile of TX x TY sites in (x, y) and a chunk of CZ planes
// in z.  It streams the planes of its tile plus a G-wide halo (G = ghost
// width >= K) through shared memory:
//   * TMA (cp.async.bulk.tensor, completion on mbarriers) copies, for every
//     input plane, a 32 x H box (H = TY + 2G) of the state (rho, m, mu) and
//     of the static data (6 hop-weight planes as one 4-D box, R) into rings
//     of shared-memory slots, P = 2 planes ahead of their first use;
//   * level j (j = 1..K) of the time block is computed one plane behind
//     level j-1 (a wavefront in z) on a region that shrinks by one site per
//     level, so the last level is exact on the core;
//   * levels 1..K-1 live in 3-plane rings in shared memory; level K is
//     written to global memory, with its ghost images.
// x neighbours come from warp shuffles (a warp is one 32-site row of the
// box), y and z neighbours from shared memory.  Per-site arithmetic is the
// same function as in the one-step kernel, so states are bit-identical to
// K launches of it.  FID / population / MSD sums of every level cover core
// sites of core planes only, so each site counts once per step.
// Every mbarrier wait is bounded; on expiry the kernel records
// LPC_ERR_TIMEOUT in the lattice's error word, waits (bounded) for its
// copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lpc_internal.cuh"
#include "tma_ptx.cuh"

namespace lpc {

namespace {

constexpr int kW = 32;      // box width (one warp per row)
constexpr int kNW = 16;     // warps per CTA
constexpr int kP = 2;       // prefetch distance in planes
constexpr int kS0 = kP + 4; // level-0 state slots (planes t-4 .. t+P-1 live)
constexpr int kRing = 4;    // planes per intermediate-level ring

constexpr int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

}  // namespace


// Geometry of one TB launch (identical in host and device).
struct TBGeom {
    int G, TX, TY, H, cz;
    int tiles_x, tiles_y, n_items;
    int state_bytes_plane;    // TMA bytes of one state plane
    int static_bytes_plane;   // TMA bytes of one static plane
    unsigned int* err;        // error word (LPC_ERR_TIMEOUT on a wait that ran out)
};

struct TBLayout {
    size_t state_slot, static_slot, off_lj, off_st, off_bar, off_red, total;
};

__host__ __device__ inline TBLayout tb_layout(int H, int K, int nmsd, int wb, int SS) {
    TBLayout L;
    const size_t plane = (size_t)H * kW;
    L.state_slot = plane * (12 + 4 * (size_t)nmsd);
    L.static_slot = plane * (6 * (size_t)wb + 8);
    L.off_lj = (size_t)kS0 * L.state_slot;
    L.off_st = L.off_lj + kRing * (size_t)(K - 1) * L.state_slot;
    L.off_bar = L.off_st + (size_t)SS * L.static_slot;
    L.off_red = L.off_bar + ((size_t)(kS0 + SS) * 8 + 15) / 16 * 16;
    L.total = L.off_red + (size_t)kNW * K * kNumSums * 8 + 128;
    return L;
}

namespace {

// Pointers into one state slot.
struct Slot {
    float* r;
    float2* m;
    float* mu[3];
};

__device__ __forceinline__ Slot slot_at(unsigned char* base, size_t slot_bytes, int plane, int nmsd) {
    Slot s;
    s.r = reinterpret_cast<float*>(base);
    s.m = reinterpret_cast<float2*>(base + (size_t)plane * 4);
    for (int a = 0; a < 3; ++a)
        s.mu[a] = a < nmsd ? reinterpret_cast<float*>(base + (size_t)plane * (12 + 4 * a)) : nullptr;
    (void)slot_bytes;
    return s;
}

template <typename WT, int K, int MSD>
__global__ void __launch_bounds__(kNW * 32, 1)
k_step_tb(const __grid_constant__ TBMaps maps, LatticeView v, TBGeom g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: round the dynamic base up
    unsigned char* smem = smem_raw + ((128u - (sa(smem_raw) & 127u)) & 127u);
    constexpr int NMSD = popc3(MSD);
    constexpr int SS = 2 * K + kP + 2;   // static planes t-2K-2 .. t+P-1 live
    const int H = g.H, G = g.G, TX = g.TX, TY = g.TY;
    const int plane = H * kW;
    const TBLayout L = tb_layout(H, K, NMSD, (int)sizeof(WT), SS);
    uint64_t* bar_s = reinterpret_cast<uint64_t*>(smem + L.off_bar);
    uint64_t* bar_w = bar_s + kS0;
    double* red = reinterpret_cast<double*>(smem + L.off_red);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < kS0; ++s) mbar_init(&bar_s[s], 1);
        for (int s = 0; s < SS; ++s) mbar_init(&bar_w[s], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < kNW * K * kNumSums; i += kNW * 32) red[i] = 0.0;
    __syncthreads();

    // axis index of the n-th enabled MSD component
    int axis_of[3] = {0, 0, 0};
    {
        int n = 0;
        for (int a = 0; a < 3; ++a)
            if (MSD >> a & 1) axis_of[n++] = a;
    }

    unsigned int issued_base = 0;    // planes loaded by this CTA before the current item
    bool failed = false;
    int fail_t = 0, fail_NQ = 0;
    const long long zplane = (long long)v.Xp * v.Yp;

    for (int item = blockIdx.x; item < g.n_items; item += gridDim.x) {
        const int tx = item % g.tiles_x;
        const int rest = item / g.tiles_x;
        const int ty = rest % g.tiles_y;
        const int zc = rest / g.tiles_y;
        const int x0 = tx * TX, y0 = ty * TY;
        const int z0 = zc * g.cz;
        const int z1 = min(z0 + g.cz, v.nz);
        const int CZ = z1 - z0;
        const int NQ = CZ + 2 * K;      // input planes of this item
        const int T = CZ + 3 * K;       // iterations (level j lags 2j planes)

        auto issue = [&](int q) {
            const unsigned int l = issued_base + q;
            int z = (z0 - K + q) % v.nz;
            if (z < 0) z += v.nz;
            unsigned char* st = smem + (size_t)(l % kS0) * L.state_slot;
            unsigned char* sw = smem + L.off_st + (size_t)(l % SS) * L.static_slot;
            uint64_t* bs = &bar_s[l % kS0];
            uint64_t* bw = &bar_w[l % SS];
            // box origin in padded coordinates: interior (x0 - G, y0 - G)
            mbar_expect_tx(bs, (uint32_t)g.state_bytes_plane);
            tma3(st, &maps.rho, bs, x0, y0, z);
            tma3(st + (size_t)plane * 4, &maps.m, bs, 2 * x0, y0, z);
#pragma unroll
            for (int a = 0; a < NMSD; ++a) tma3(st + (size_t)plane * (12 + 4 * a), &maps.mu[a], bs, x0, y0, z);
            mbar_expect_tx(bw, (uint32_t)g.static_bytes_plane);
            tma4(sw, &maps.w, bw, x0, y0, z, 0);
            tma3(sw + (size_t)plane * 6 * sizeof(WT), &maps.R, bw, 2 * x0, y0, z);
        };

        if (tid == 0) {
            fence_proxy_async();
            for (int q = 0; q < kP && q < NQ; ++q) issue(q);
        }
        // per-thread FP32 sums of each level over this item's core sites
        float part[K][kNumSums];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int qq = 0; qq < kNumSums; ++qq) part[j][qq] = 0.f;

        for (int t = 0; t < T; ++t) {
            if (tid == 0 && t + kP < NQ) {
                fence_proxy_async();
                issue(t + kP);
            }
            // this iteration reads input planes up to t-1
            bool ok = true;
            if (t >= 1 && t - 1 < NQ) {
                const unsigned int l = issued_base + (t - 1);
                ok = mbar_wait_bounded(&bar_s[l % kS0], (l / kS0) & 1u);
                ok = ok && mbar_wait_bounded(&bar_w[l % SS], (l / SS) & 1u);
            }
            // tasks of this iteration: (level j, row) for every active level;
            // level j computes plane q = t - 2j, so no level reads a plane
            // written in the same iteration
            int cnt[K];
            int ntask = 0;
#pragma unroll
            for (int j = 1; j <= K; ++j) {
                const int q = t - 2 * j;
                cnt[j - 1] = (q >= j && q <= NQ - 1 - j) ? TY + 2 * (K - j) : 0;
                ntask += cnt[j - 1];
            }
            for (int task = warp; task < ntask; task += kNW) {
                int j = 1, r = task;
#pragma unroll
                for (int jj = 0; jj < K - 1; ++jj)
                    if (j == jj + 1 && r >= cnt[jj]) { r -= cnt[jj]; j = jj + 2; }
                const int lo = G - K + j;
                r += lo;                                  // box row
                const int q = t - 2 * j;                  // chunk-relative plane
                Slot in[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const int qq = q - 1 + d;
                    unsigned char* base;
                    if (j == 1) base = smem + (size_t)((issued_base + qq) % kS0) * L.state_slot;
                    else base = smem + L.off_lj + ((size_t)(j - 2) * kRing + (qq % kRing)) * L.state_slot;
                    in[d] = slot_at(base, L.state_slot, plane, NMSD);
                }
                const WT* ws[3];
                const float2* Rq = nullptr;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    unsigned char* bp = smem + L.off_st + (size_t)((issued_base + q - 1 + d) % SS) * L.static_slot;
                    ws[d] = reinterpret_cast<const WT*>(bp);
                    if (d == 1) Rq = reinterpret_cast<const float2*>(bp + (size_t)plane * 6 * sizeof(WT));
                }
                const int hic = G + TX + K - j;           // end column of this level
                const int zl = z0 - K + q;                // lattice plane (unwrapped)
                const bool core_plane = zl >= z0 && zl < z1;
                const bool active_c = lane >= lo && lane < hic;
                const bool core_c = lane >= G && lane < G + TX && (x0 + lane - G) < v.nx;
                const int o = r * kW + lane;
                SiteIn qi;
                float wo[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) wo[k] = lds_w<WT>(ws[1] + k * plane + o);
                qi.rc = in[1].r[o];
                qi.mc = in[1].m[o];
                qi.r[0] = __shfl_up_sync(0xffffffffu, qi.rc, 1);
                qi.m[0].x = __shfl_up_sync(0xffffffffu, qi.mc.x, 1);
                qi.m[0].y = __shfl_up_sync(0xffffffffu, qi.mc.y, 1);
                qi.win[0] = __shfl_up_sync(0xffffffffu, wo[0], 1);
                qi.r[1] = __shfl_down_sync(0xffffffffu, qi.rc, 1);
                qi.m[1].x = __shfl_down_sync(0xffffffffu, qi.mc.x, 1);
                qi.m[1].y = __shfl_down_sync(0xffffffffu, qi.mc.y, 1);
                qi.win[1] = __shfl_down_sync(0xffffffffu, wo[1], 1);
                qi.r[2] = in[1].r[o - kW];
                qi.m[2] = in[1].m[o - kW];
                qi.win[2] = lds_w<WT>(ws[1] + 2 * plane + o - kW);
                qi.r[3] = in[1].r[o + kW];
                qi.m[3] = in[1].m[o + kW];
                qi.win[3] = lds_w<WT>(ws[1] + 3 * plane + o + kW);
                qi.r[4] = in[0].r[o];
                qi.m[4] = in[0].m[o];
                qi.win[4] = lds_w<WT>(ws[0] + 4 * plane + o);
                qi.r[5] = in[2].r[o];
                qi.m[5] = in[2].m[o];
                qi.win[5] = lds_w<WT>(ws[2] + 5 * plane + o);
#pragma unroll
                for (int k = 0; k < 6; ++k) qi.wout[k] = wo[k];
                qi.R = Rq[o];
                const float s = stay_weight(wo);
                float ro;
                float2 mo;
                site_rho_m(qi, s, ro, mo);
                float muo[3] = {0.f, 0.f, 0.f}, dms[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int n = 0; n < NMSD; ++n) {
                    const int a = axis_of[n];
                    const float muc = in[1].mu[n][o];
                    float nb[6];
                    nb[0] = __shfl_up_sync(0xffffffffu, muc, 1);
                    nb[1] = __shfl_down_sync(0xffffffffu, muc, 1);
                    nb[2] = in[1].mu[n][o - kW];
                    nb[3] = in[1].mu[n][o + kW];
                    nb[4] = in[0].mu[n][o];
                    nb[5] = in[2].mu[n][o];
                    muo[n] = site_mu(qi.win, qi.r, nb, s, muc, a);
                    dms[n] = site_dmsd(wo, muc, qi.rc, a);
                }
                const bool core = core_plane && core_c && r >= G && r < G + TY && (y0 + r - G) < v.ny;
                if (active_c) {
                    if (j < K) {
                        Slot out = slot_at(smem + L.off_lj + ((size_t)(j - 1) * kRing + (q % kRing)) * L.state_slot,
                                           L.state_slot, plane, NMSD);
                        out.r[o] = ro;
                        out.m[o] = mo;
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) out.mu[n][o] = muo[n];
                    } else if (core) {
                        const int x = x0 + lane - G, y = y0 + r - G;
                        const long long zoff = (long long)zl * zplane;
                        store_images(v.rho_out, v, x, y, zoff, ro);
                        store_images(v.m_out, v, x, y, zoff, mo);
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) store_images(v.mu_out[axis_of[n]], v, x, y, zoff, muo[n]);
                    }
                }
                if (core) {
#pragma unroll
                    for (int jj = 0; jj < K; ++jj)
                        if (jj == j - 1) {
                            part[jj][0] += mo.x;
                            part[jj][1] += mo.y;
                            part[jj][2] += ro;
#pragma unroll
                            for (int n = 0; n < NMSD; ++n) part[jj][3 + axis_of[n]] += dms[n];
                        }
                }
            }
            if (__syncthreads_or(!ok)) {
                failed = true;
                fail_t = t;
                fail_NQ = NQ;
                break;
            }
        }
        if (failed) break;
        // one FP32 warp reduction per level and quantity per item, FP64 per warp
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double* acc = red + ((size_t)j * kNW + warp) * kNumSums;
#pragma unroll
            for (int qq = 0; qq < kNumSums; ++qq) {
                if (qq >= 3 && !(MSD >> (qq - 3) & 1)) continue;
                const float tsum = warp_sum_f32(part[j][qq]);
                if (lane == 0) acc[qq] += (double)tsum;
            }
        }
        issued_base += (unsigned int)NQ;
    }

    if (failed) {
        // record the timeout, then wait (bounded) for the copies still in flight
        if (tid == 0) {
            atomicExch(g.err, (unsigned int)LPC_ERR_TIMEOUT);
            const int first = fail_t >= 1 ? fail_t - 1 : 0;
            const int last = min(fail_t + kP, fail_NQ);
            for (int q = first; q < last; ++q) {
                const unsigned int l = issued_base + q;
                mbar_wait_bounded(&bar_s[l % kS0], (l / kS0) & 1u);
                mbar_wait_bounded(&bar_w[l % SS], (l / SS) & 1u);
            }
        }
        __syncthreads();
        return;
    }
    block_finish_smem<kNW>(v, K, red);
}

template <typename WT, int K, int MSD>
void* tb_fn() { return reinterpret_cast<void*>(&k_step_tb<WT, K, MSD>); }

template <typename WT, int K>
void* tb_fn_msd(int msd) {
    switch (msd & 7) {
        case 0: return tb_fn<WT, K, 0>();
        case 1: return tb_fn<WT, K, 1>();
        case 2: return tb_fn<WT, K, 2>();
        case 3: return tb_fn<WT, K, 3>();
        case 4: return tb_fn<WT, K, 4>();
        case 5: return tb_fn<WT, K, 5>();
        case 6: return tb_fn<WT, K, 6>();
        default: return tb_fn<WT, K, 7>();
    }
}

template <typename WT>
void* tb_fn_k(int K, int msd) {
    switch (K) {
        case 1: return tb_fn_msd<WT, 1>(msd);
        case 2: return tb_fn_msd<WT, 2>(msd);
        case 3: return tb_fn_msd<WT, 3>(msd);
        default: return tb_fn_msd<WT, 4>(msd);
    }
}

void* tb_kernel(int wdtype, int K, int msd) {
    return wdtype == LPC_WEIGHTS_BF16 ? tb_fn_k<__nv_bfloat16>(K, msd) : tb_fn_k<float>(K, msd);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool tma_encode(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}


// Column alignment of a TMA box start: 16 bytes of the narrowest element.
static int tb_align(int wdtype) { return wdtype == LPC_WEIGHTS_BF16 ? 8 : 4; }

bool tb_supported(const LatticeView& v, int wdtype, int K) {
    if (K == 1) return t1_supported(v, wdtype);
    if (K < 1 || K > 4 || K > v.G) return false;
    const int TX = (kW - 2 * v.G) / tb_align(wdtype) * tb_align(wdtype);
    return TX >= tb_align(wdtype) && encode_fn() != nullptr;
}

int tb_plan(const LatticeView& v, int wdtype, int K, TBGeom* out) {
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    const int nmsd = popc3(v.msd_axes);
    const int SS = 2 * K + kP + 2;
    const int A = tb_align(wdtype);
    TBGeom g{};
    g.G = v.G;
    g.TX = (kW - 2 * v.G) / A * A;
    const size_t budget = (size_t)device_props().max_smem_optin - 1024;   // static smem margin
    int H = 2 * v.G + 1;
    for (int h = 2 * v.G + 1; h <= 64; ++h)
        if (tb_layout(h, K, nmsd, wb, SS).total <= budget) H = h;
    if (tb_layout(H, K, nmsd, wb, SS).total > budget) return -1;
    g.H = H;
    g.TY = H - 2 * v.G;
    g.tiles_x = (v.nx + g.TX - 1) / g.TX;
    g.tiles_y = (v.ny + g.TY - 1) / g.TY;
    const long long xy = (long long)g.tiles_x * g.tiles_y;
    const int sms = device_props().sm_count;
    // z chunks: at least ~8 items per SM, chunks of >= 8K planes when possible
    long long nchunks = (8LL * sms + xy - 1) / xy;
    int cz = (int)((v.nz + nchunks - 1) / nchunks);
    if (cz < 8 * K) cz = 8 * K;
    if (cz > v.nz) cz = v.nz;
    g.cz = cz;
    g.n_items = (int)(xy * ((v.nz + cz - 1) / cz));
    g.state_bytes_plane = H * kW * (12 + 4 * nmsd);
    g.static_bytes_plane = H * kW * (6 * wb + 8);
    *out = g;
    return (int)tb_layout(H, K, nmsd, wb, SS).total;
}

bool tb_encode_maps(const LatticeView& v, int wdtype, int W, int H, TBMaps* maps) {
    const cuuint64_t Xp = (cuuint64_t)v.Xp, Yp = (cuuint64_t)v.Yp, nz = (cuuint64_t)v.nz;
    const cuuint32_t Hb = (cuuint32_t)H;
    bool ok = true;
    {
        const cuuint64_t dims[3] = {Xp, Yp, nz};
        const cuuint64_t str[2] = {Xp * 4, Xp * Yp * 4};
        const cuuint32_t box[3] = {(cuuint32_t)W, Hb, 1};
        ok = ok && tma_encode(&maps->rho, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.rho_in, dims, str, box);
        for (int a = 0, n = 0; a < 3; ++a)
            if (v.msd_axes >> a & 1) ok = ok && tma_encode(&maps->mu[n++], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.mu_in[a], dims, str, box);
    }
    {
        const cuuint64_t dims[3] = {2 * Xp, Yp, nz};
        const cuuint64_t str[2] = {2 * Xp * 4, 2 * Xp * Yp * 4};
        const cuuint32_t box[3] = {(cuuint32_t)(2 * W), Hb, 1};
        ok = ok && tma_encode(&maps->m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.m_in, dims, str, box);
        ok = ok && tma_encode(&maps->R, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.R, dims, str, box);
    }
    {
        const cuuint64_t e = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
        const cuuint64_t dims[4] = {Xp, Yp, nz, 6};
        const cuuint64_t str[3] = {Xp * e, Xp * Yp * e, (cuuint64_t)v.Np * e};
        const cuuint32_t box[4] = {(cuuint32_t)W, Hb, 1, 6};
        ok = ok && tma_encode(&maps->w, wdtype == LPC_WEIGHTS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          4, v.w, dims, str, box);
    }
    return ok;
}

cudaError_t tb_prepare(int wdtype, int K, int msd) {
    if (K == 1) return t1_prepare(wdtype, msd);
    // opt in to the large dynamic shared memory once per kernel (host only,
    // called before any stream capture)
    static bool attr_set[2][5][8] = {};
    bool& done = attr_set[wdtype == LPC_WEIGHTS_BF16][K][msd & 7];
    if (done) return cudaSuccess;
    void* fn = tb_kernel(wdtype, K, msd);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    // the opt-in limit covers static + dynamic shared memory
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             device_props().max_smem_optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_tb(const LatticeView& v, int wdtype, int K, const TBMaps& maps, unsigned int* err,
                      cudaStream_t st) {
    if (K == 1) return launch_tma1(v, wdtype, maps, err, st);
    TBGeom g;
    const int smem = tb_plan(v, wdtype, K, &g);
    if (smem < 0) return cudaErrorInvalidConfiguration;
    g.err = err;
    void* fn = tb_kernel(wdtype, K, v.msd_axes);
    cudaError_t e0 = tb_prepare(wdtype, K, v.msd_axes);
    if (e0 != cudaSuccess) return e0;
    int grid = device_props().sm_count;
    if (grid > g.n_items) grid = g.n_items;
    LatticeView vv = v;
    TBMaps mm = maps;
    void* args[] = {&mm, &vv, &g};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kNW * 32), args, (size_t)smem, st);
}

bool tb_box_dims(const LatticeView& v, int wdtype, int K, int* W, int* H) {
    TBGeom g;
    if (tb_plan(v, wdtype, K, &g) < 0) return false;
    *W = kW;
    *H = g.H;
    return true;
}

size_t tb_maps_size() { return sizeof(TBMaps); }
TBMaps* tb_maps_new() { return new TBMaps(); }
void tb_maps_delete(TBMaps* m) { delete m; }

int tb_grid(const LatticeView& v, int wdtype, int K) {
    TBGeom g;
    if (tb_plan(v, wdtype, K, &g) < 0) return 0;
    const int sms = device_props().sm_count;
    return g.n_items < sms ? g.n_items : sms;
}

}  // namespace lpc
