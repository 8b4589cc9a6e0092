// One time step per launch fed by TMA with warp specialisation (the TB
// schedule at block depth 1).
//
// Work items are (z-chunk, tile) pairs, tile index fastest, taken from a
// global queue (one atomic per item) by a persistent grid of one CTA per SM,
// so that CTAs that run slower take fewer items and neighbouring tiles are
// in flight at the same time.  A tile is 64 x TY (x, y) sites: TY consumer
// warps, one row each, two neighbouring x sites per lane.  An item streams
// the planes za-1 .. zb of its z-chunk.
//
// A producer lane fills two rings of shared-memory slots with
// cp.async.bulk.tensor:
//   state  (S1 slots): rho, m, mu of one plane, W = 64 + 2G columns
//          (rounded up to 16 bytes, from the aligned ghost column of a
//          128-byte-aligned row) x TY + 2 rows: the x and y neighbours that
//          the gather reads;
//   static (S2 slots): the gather form of the static data of one plane's
//          core (in-weights of the six incoming hops, stay weight, rotation,
//          MSD out-weights), 64 x TY, no halo, rows on 256-byte boundaries.
// Each slot has a "full" mbarrier (TMA transaction bytes) and an "empty"
// mbarrier (one arrival per consumer warp); state slots carry a header with
// the item, so the consumers follow the producer through the queue.  A
// consumer warp waits for the static data of the centre plane and the state
// of the plane above, updates its two sites per lane (the plane below is
// kept in registers) and releases both.  A header with a negative tile ends
// the launch.  Per-site arithmetic is the shared site function with the same
// FP32 in-weights and stay weight, so states are bit-identical to the other
// kernels.
//
// Every wait is bounded (clock64 budget); on expiry the kernel records
// LPC_ERR_TIMEOUT in the lattice's error word, waits (bounded) for its
// copies in flight and returns without writing the step's sums.
#include "lpc_internal.cuh"
#include "tma_ptx.cuh"

#ifndef LPC_T1_MIN_DEPTH
#define LPC_T1_MIN_DEPTH 3
#endif
#ifndef LPC_T1_ITEMS_PER_CTA
#define LPC_T1_ITEMS_PER_CTA 40
#endif

namespace lpc {

namespace {

constexpr int kTX = 64;      // core columns of a tile
constexpr int popc(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }

// Position in a slot ring: slot index and the parity of its barrier phase.
struct Cursor {
    int slot;
    unsigned int ph;
    __device__ __forceinline__ void next(int S) {
        if (++slot == S) { slot = 0; ph ^= 1u; }
    }
};

// Two consecutive in-weights in shared memory as floats.
template <typename WT> __device__ __forceinline__ float2 lds_w2(const WT* p);
template <> __device__ __forceinline__ float2 lds_w2<float>(const float* p) {
    return *reinterpret_cast<const float2*>(p);
}
template <> __device__ __forceinline__ float2 lds_w2<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned int u = *reinterpret_cast<const unsigned int*>(p);
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// Four consecutive weights in shared memory as floats.
template <typename WT> __device__ __forceinline__ float4 lds_w4(const WT* p);
template <> __device__ __forceinline__ float4 lds_w4<float>(const float* p) {
    return *reinterpret_cast<const float4*>(p);
}
template <> __device__ __forceinline__ float4 lds_w4<__nv_bfloat16>(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

}  // namespace

struct T1Geom {
    int W, TY, S1, S2;
    int dm_src;                 // stage the MSD out-weight pairs (source-attributed MSD sums)
    int tiles_x, tiles, cz, n_items;
    int slot1, slot2;           // bytes of a state / static slot
    int tx1, tx2;               // transaction bytes of a state / static load
    unsigned int* err;
    unsigned int* work;
    float abig;                 // link form: the weight of a downhill or level hop, alpha/6 as stored
};

namespace {

// state slot:  rho [TY+2][W] f32 | m [TY+2][W] f32x2 | mu_n [TY+2][W] f32
// static slot, gather form: win [6][TY][64] WT | s [TY][64] f32 | R [TY][64] f32x2
//              | dm_n [TY][64] WTx2 (pairs of MSD axes y, z) | dx [TY] WTx2 (x out-weights
//              at the tile's ends) | lab [TY][64] u8 (region labels, with regions only)
// static slot, link form:   lx [TY][64] WT | ly [TY+1][64] WT (the row above too) | lz [TY][64] WT
//              | R [TY][64] f32x2
// (each part on a 128-byte boundary, as TMA requires)
struct T1Slots {
    int m, mu[3], bytes1;
    int s, R, dm[3], dx, lab, bytes2;
    int lx, ly, lz;
};
__host__ __device__ inline int up128(int n) { return (n + 127) / 128 * 128; }
// MSD sums over source sites (regions, reservoir faces: src) take every
// site's out-weights of each MSD axis.  Those of x come from the x
// neighbours' in-weights, which the gather holds, and from the tile-edge
// array; those of y and z are staged as pairs.  Returned: the bitmask, over
// the index n of the MSD axes in order, of the staged pairs.
__host__ __device__ inline int t1_dm_staged(int msd, bool src) {
    if (!src) return 0;
    const int nmsd = (msd & 1) + ((msd >> 1) & 1) + ((msd >> 2) & 1);
    return ((1 << nmsd) - 1) & ~(msd & 1);
}
// dmn: t1_dm_staged; dmx: the tile-edge x out-weights are staged
__host__ __device__ inline T1Slots t1_slots(int W, int TY, int nmsd, int wb, bool rho_only, bool reg, int dmn,
                                            bool dmx, bool lnk = false) {
    T1Slots L;
    const int H = TY + 2;
    int off = up128(H * W * 4);
    L.m = off;
    if (!rho_only) off += up128(H * W * 8);
    for (int n = 0; n < 3; ++n) {
        L.mu[n] = off;
        if (n < nmsd) off += up128(H * W * 4);
    }
    L.bytes1 = off;
    const int C = TY * kTX;
    if (lnk) {
        L.lx = 0;
        off = up128(C * wb);
        L.ly = off;
        off += up128(C * wb + kTX * wb);
        L.lz = off;
        off += up128(C * wb);
        L.R = off;
        if (!rho_only) off += up128(C * 8);
        L.s = off;
        for (int n = 0; n < 3; ++n) L.dm[n] = off;
        L.dx = off;
        L.lab = off;
        if (reg) off += up128(C);
        L.bytes2 = off;
        return L;
    }
    L.lx = L.ly = L.lz = 0;
    off = up128(6 * C * wb);
    L.s = off;
    off += up128(C * 4);
    L.R = off;
    if (!rho_only) off += up128(C * 8);
    for (int n = 0; n < 3; ++n) {
        L.dm[n] = off;
        if (dmn >> n & 1) off += up128(C * 2 * wb);
    }
    L.dx = off;
    if (dmx) off += up128(TY * 2 * wb);
    L.lab = off;
    if (reg) off += up128(C);
    L.bytes2 = off;
    return L;
}

// Per-item sums: the totals, and with regions each region's (KS values,
// stored with a stride of KSP doubles per warp in shared memory).
template <bool REG> struct ItemSums {
    static constexpr int KS = REG ? kNumSums * (1 + LPC_MAX_REGIONS) : kNumSums;
    static constexpr int KSP = REG ? 32 : 8;
};

struct SlotHdr {
    int tile, za, n, pad;
};

// Link form (LNK): the static data of a plain lattice (one jump factor,
// no reservoir face, no regions) as one signed value per link and axis,
// L_a(y) for the link between y and y + e_a: 0 = closed; L > 0: the hop
// y -> y + e_a has weight L and the hop back the weight A = alpha/6 of a
// downhill or level Metropolis move (Eq. 1); L < 0: the hop y -> y + e_a has
// weight A and the hop back -L.  One of the two hops of an open link is
// always A, so these are exactly the stored weights.  A closed link is
// stored as +0 (never -0), so one comparison per direction decides.
__device__ __forceinline__ float link_fwd(float L, float A) { return L < 0.f ? A : L; }
__device__ __forceinline__ float link_bwd(float L, float A) { return L > 0.f ? A : fabsf(L); }

template <typename WT, int MSD, int NC, bool RHO, bool REG, bool LNK>
__global__ void __launch_bounds__((NC + 1) * 32, 1)
k_step_tma1(const __grid_constant__ TBMaps maps, LatticeView v, T1Geom g) {
    static_assert(!RHO || MSD == 0, "the rho-only step carries no moments");
    static_assert(!RHO || !REG, "the rho-only step takes no sums");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (sa(smem_raw) & 127u)) & 127u);
    constexpr int NMSD = popc(MSD);
    constexpr int TY = NC;                    // one core row per consumer warp
    constexpr int KS = ItemSums<REG>::KS, KSP = ItemSums<REG>::KSP;
    static_assert(KS <= 32, "one lane per item sum");
    const int W = g.W, S1 = g.S1, S2 = g.S2;
    // MSD increments: summed over the source sites with their out-weights
    // where regions or reservoir faces need that attribution (x from the
    // neighbours' in-weights and the tile-edge values, y and z from staged
    // pairs), else over the destination sites with the in-weights and source
    // states the gather already holds (the same total, without the pairs)
    const bool src_msd = !LNK && (REG || g.dm_src);
    const int dmn = t1_dm_staged(MSD, src_msd);
    const bool dmx = src_msd && (MSD & 1);
    const T1Slots SL = t1_slots(W, TY, NMSD, (int)sizeof(WT), RHO, REG, dmn, dmx, LNK);
    unsigned char* ring1 = smem;
    unsigned char* ring2 = smem + (size_t)S1 * g.slot1;
    uint64_t* full1 = reinterpret_cast<uint64_t*>(ring2 + (size_t)S2 * g.slot2);
    uint64_t* empty1 = full1 + S1;
    uint64_t* full2 = empty1 + S1;
    uint64_t* empty2 = full2 + S2;
    uint64_t* ifree = empty2 + S2;                                  // [2] item sums combined
    unsigned int* icount = reinterpret_cast<unsigned int*>(ifree + 2);   // [2] warps done
    SlotHdr* hdr = reinterpret_cast<SlotHdr*>(ifree + 3);          // [S1]
    double* ired = reinterpret_cast<double*>(hdr + S1);            // [2][NC][KSP] per-warp item sums
    volatile int* abort_flag = reinterpret_cast<volatile int*>(ired + 2 * NC * KSP);
    volatile unsigned int* issued1 = reinterpret_cast<volatile unsigned int*>(abort_flag + 1);
    volatile unsigned int* issued2 = issued1 + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = v.G;
    const int nz = v.nz;

    if (tid == 0) {
        for (int s = 0; s < S1; ++s) {
            mbar_init(&full1[s], 1);
            mbar_init(&empty1[s], NC);
        }
        for (int s = 0; s < S2; ++s) {
            mbar_init(&full2[s], 1);
            mbar_init(&empty2[s], NC);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ifree[b], 1);
            icount[b] = 0u;
        }
        *abort_flag = 0;
        *issued1 = 0;
        *issued2 = 0;
        fence_mbar_init();
    }
    __syncthreads();

    int axis_of[3] = {0, 0, 0};
    {
        int n = 0;
        for (int a = 0; a < 3; ++a)
            if (MSD >> a & 1) axis_of[n++] = a;
    }

    if (warp == NC) {
        // ---------------- producer warp: one elected lane takes items and issues the copies
        if (lane == 0) {
            bool ok = true;
            Cursor c1{0, 0u}, c2{0, 0u};
            unsigned int n1 = 0, n2 = 0;
            // one state load (plane z of the item) with its header
            auto state_load = [&](int z, const SlotHdr& h, int bx, int by) -> bool {
                if (n1 >= (unsigned)S1 && !mbar_wait_bounded(&empty1[c1.slot], c1.ph ^ 1u)) return false;
                if (*abort_flag) return false;
                hdr[c1.slot] = h;
                unsigned char* st = ring1 + (size_t)c1.slot * g.slot1;
                uint64_t* fb = &full1[c1.slot];
                fence_proxy_async();
                if (h.tile < 0) {
                    mbar_arrive(fb);                  // end marker: no copy
                } else {
                    mbar_expect_tx(fb, (uint32_t)g.tx1);
                    tma3(st, &maps.rho, fb, bx, by, z);
                    if (!RHO) tma3(st + SL.m, &maps.m, fb, 2 * bx, by, z);
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) tma3(st + SL.mu[n], &maps.mu[n], fb, bx, by, z);
                }
                *issued1 = ++n1;
                c1.next(S1);
                return true;
            };
            for (;;) {
                const int item = (int)atomicAdd(g.work, 1u);
                if (item >= g.n_items) break;
                const int tile = item % g.tiles;
                const int za = v.zlo + (item / g.tiles) * g.cz;
                const int n = min(g.cz, v.zhi - za);
                const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
                const int bx = tx * kTX;                 // padded column of the state box
                const int by = ty * TY + G - 1;          // padded row of y0 - 1
                const int sx = tx * kTX, sy = ty * TY;   // gather-form box origin
                const SlotHdr h{tile, za, n, 0};
                ok = state_load(za == 0 ? nz - 1 : za - 1, h, bx, by) && state_load(za, h, bx, by);
                for (int q = 0; q < n && ok; ++q) {
                    // static data of centre za + q, then the state of the plane above it
                    if (n2 >= (unsigned)S2) ok = mbar_wait_bounded(&empty2[c2.slot], c2.ph ^ 1u);
                    if (!ok || *abort_flag) { ok = false; break; }
                    {
                        unsigned char* st = ring2 + (size_t)c2.slot * g.slot2;
                        uint64_t* fb = &full2[c2.slot];
                        const int z = za + q;
                        fence_proxy_async();
                        mbar_expect_tx(fb, (uint32_t)g.tx2);
                        if (LNK) {
                            // link planes in rows of ny + 1 (row 0: the image of row ny - 1)
                            tma4(st + SL.lx, &maps.glnk1, fb, sx, sy + 1, z, 0);
                            tma4(st + SL.ly, &maps.glnk2, fb, sx, sy, z, 1);
                            tma4(st + SL.lz, &maps.glnk1, fb, sx, sy + 1, z, 2);
                        } else {
                            tma4(st, &maps.gwin, fb, sx, sy, z, 0);
                            tma3(st + SL.s, &maps.gs, fb, sx, sy, z);
                        }
                        if (!RHO) tma3(st + SL.R, &maps.gR, fb, 2 * sx, sy, z);
#pragma unroll
                        for (int m = 0; m < NMSD; ++m)
                            if (dmn >> m & 1) tma4(st + SL.dm[m], &maps.gdm, fb, 2 * sx, sy, z, axis_of[m]);
                        if (dmx) tma3(st + SL.dx, &maps.gdx, fb, 2 * sy, tx, z);
                        if (REG) tma3(st + SL.lab, &maps.glab, fb, sx, sy, z);
                        *issued2 = ++n2;
                        c2.next(S2);
                    }
                    const int za1 = za + q + 1;
                    ok = state_load(za1 == nz ? 0 : za1, h, bx, by);
                }
                if (!ok) break;
            }
            if (ok) ok = state_load(0, SlotHdr{-1, 0, 0, 0}, 0, 0);
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---------------- consumer warps: core row `warp`, sites x0 + 2 lane + {0, 1}
        float part[kNumSums] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // Region sums (REG): preg[region][Mre, Mim, P, dMSD of each MSD axis in
        // order].  Regions are mostly large connected parts, so a warp's row of
        // 64 sites usually lies in one region for many planes: `part` then sums
        // the current run of planes whose row has the warp-uniform label
        // `curlab`, and is added to that region when the label changes (and at
        // the item's end, where the totals become the sum over regions).  Rows
        // that mix labels add each site to its region directly.
        float preg[REG ? LPC_MAX_REGIONS : 1][3 + NMSD];
#pragma unroll
        for (int r = 0; r < (REG ? LPC_MAX_REGIONS : 1); ++r)
#pragma unroll
            for (int q = 0; q < 3 + NMSD; ++q) preg[r][q] = 0.f;
        int curlab = -1;
        unsigned int touched = 0u;      // regions with sums in this item (warp-uniform)
        auto flush_run = [&]() {
            if (curlab >= 0) touched |= 1u << curlab;
#pragma unroll
            for (int r = 0; r < (REG ? LPC_MAX_REGIONS : 1); ++r)
                if (curlab == r) {
                    preg[r][0] += part[0];
                    preg[r][1] += part[1];
                    preg[r][2] += part[2];
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) preg[r][3 + n] += part[3 + axis_of[n]];
                }
#pragma unroll
            for (int q = 0; q < kNumSums; ++q) part[q] = 0.f;
        };
        bool ok = true;
        Cursor w1{0, 0u}, w2{0, 0u};
        unsigned int kitem = 0;                          // items this warp has finished
        const int o = (warp + 1) * W + G + 2 * lane;     // site 0 in the state arrays
        const int os = warp * kTX + 2 * lane;            // site 0 in the static arrays
        const int C = TY * kTX;
        const long long zplane = (long long)v.Xp * v.Yp;
        for (;;) {
            ok = mbar_wait_bounded(&full1[w1.slot], w1.ph);
            if (!ok) break;
            const SlotHdr h = hdr[w1.slot];
            if (h.tile < 0) break;                       // end of the queue
            const int tx = h.tile % g.tiles_x, ty = h.tile / g.tiles_x;
            const int x = tx * kTX + 2 * lane;
            const int y = ty * TY + warp;
            const bool ok_y = y < v.ny;
            const bool site0 = ok_y && x < v.nx;
            const bool site1 = ok_y && x + 1 < v.nx;
            // the pair has ghost images to write: it lies within G of a periodic face
            const bool images = (v.per_x && (x < G || x + 1 >= v.nx - G)) || (v.per_y && (y < G || y >= v.ny - G));
            const long long col = (long long)(y + G) * v.Xp + (x + G);
            // link form: the weights of the +z links of the plane below (they
            // end in this plane: in-weight along +z, out-weight along -z) and,
            // for lane 0, the +x link of the site left of the tile (it ends in
            // site 0), read from global memory; later planes take the +z
            // weights from the previous plane
            float2 zin = make_float2(0.f, 0.f), zout = make_float2(0.f, 0.f);
            float lxe = 0.f, lxe1 = 0.f;                           // lane 0: this plane's and the next
            const WT* lnk = static_cast<const WT*>(v.lnk);
            const long long lplane = (long long)v.ny1 * v.Xs;     // one axis, one plane
            // lane 0: the +x link that ends in site 0, from the column left of
            // the tile (at x = 0 the links that enter column 0 from the left)
            const WT* lx0 = static_cast<const WT*>(v.lnk_x0);
            auto left_link = [&](int zz) -> float {
                return x == 0 ? ldw<WT>(lx0 + (long long)zz * v.ny + y)
                              : ldw<WT>(lnk + (long long)zz * lplane + (long long)(y + 1) * v.Xs + x - 1);
            };
            if (LNK) {
                const int zb = h.za == 0 ? nz - 1 : h.za - 1;
                const long long lb = (2LL * nz + zb) * lplane + (long long)(y + 1) * v.Xs + x;
                const float lzb0 = site0 ? ldw<WT>(lnk + lb) : 0.f;
                const float lzb1 = site1 ? ldw<WT>(lnk + lb + 1) : 0.f;
                zin = make_float2(link_fwd(lzb0, g.abig), link_fwd(lzb1, g.abig));
                zout = make_float2(link_bwd(lzb0, g.abig), link_bwd(lzb1, g.abig));
                if (lane == 0 && ok_y) {
                    lxe = left_link(h.za);
                    if (h.n > 1) lxe1 = left_link(h.za + 1);
                }
            }
            // plane za-1: keep this lane's two columns as "below"
            float2 br, bmu[3];
            float4 bm;
            {
                const unsigned char* s0 = ring1 + (size_t)w1.slot * g.slot1;
                br = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(s0) + o);
                if (!RHO) bm = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(s0 + SL.m) + o);
#pragma unroll
                for (int n = 0; n < NMSD; ++n)
                    bmu[n] = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(s0 + SL.mu[n]) + o);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty1[w1.slot]);
                w1.next(S1);
            }
            // plane za: the first centre
            ok = mbar_wait_bounded(&full1[w1.slot], w1.ph);
            int center = w1.slot;
            w1.next(S1);
            for (int q = 0; q < h.n && ok; ++q) {
                const int z = h.za + q;
                const int sslot = w2.slot;
                ok = mbar_wait_bounded(&full2[sslot], w2.ph);
                w2.next(S2);
                const int above = w1.slot;
                ok = ok && mbar_wait_bounded(&full1[above], w1.ph);
                w1.next(S1);
                if (!ok || *abort_flag) { ok = false; break; }
                const unsigned char* sc = ring1 + (size_t)center * g.slot1;
                const unsigned char* sv = ring1 + (size_t)above * g.slot1;
                const unsigned char* ss = ring2 + (size_t)sslot * g.slot2;
                const float* rc = reinterpret_cast<const float*>(sc);
                const float2 r_c = *reinterpret_cast<const float2*>(rc + o);
                const float r_l = rc[o - 1], r_r = rc[o + 2];
                const float2 r_u = *reinterpret_cast<const float2*>(rc + o - W);
                const float2 r_d = *reinterpret_cast<const float2*>(rc + o + W);
                const float2 r_a = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sv) + o);
                float2 muc[3];
#pragma unroll
                for (int n = 0; n < NMSD; ++n)
                    muc[n] = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sc + SL.mu[n]) + o);

                SiteIn q0, q1;
                float2 sp;
                float2 win2[6];                  // in-weights of the two sites (.x site 0, .y site 1)
                float2 wo2[6];                   // link form: their out-weights
                float lwo0[6], lwo1[6];
                if constexpr (LNK) {
                    const float A = g.abig;
                    const float2 lx = lds_w2<WT>(reinterpret_cast<const WT*>(ss + SL.lx) + os);
                    const float2 lyb = lds_w2<WT>(reinterpret_cast<const WT*>(ss + SL.ly) + os);       // row above
                    const float2 ly = lds_w2<WT>(reinterpret_cast<const WT*>(ss + SL.ly) + os + kTX);  // own row
                    const float2 lz = lds_w2<WT>(reinterpret_cast<const WT*>(ss + SL.lz) + os);
                    float lxm = __shfl_up_sync(0xffffffffu, lx.y, 1);   // +x link ending in site 0
                    if (lane == 0) lxm = lxe;
                    // each link's two weights: forward (+a) and backward (-a)
                    const float xf = link_fwd(lx.x, A), xb = link_bwd(lx.x, A);
                    const float2 zf = make_float2(link_fwd(lz.x, A), link_fwd(lz.y, A));
                    const float2 zb = make_float2(link_bwd(lz.x, A), link_bwd(lz.y, A));
                    // in-weights: the +a hop from y - e_a, the -a hop back over y's own link
                    win2[0] = make_float2(link_fwd(lxm, A), xf);
                    win2[1] = make_float2(xb, link_bwd(lx.y, A));
                    win2[2] = make_float2(link_fwd(lyb.x, A), link_fwd(lyb.y, A));
                    win2[3] = make_float2(link_bwd(ly.x, A), link_bwd(ly.y, A));
                    win2[4] = zin;
                    win2[5] = zb;
                    // out-weights: forward over the own link, backward over y - e_a's
                    wo2[0] = make_float2(xf, link_fwd(lx.y, A));
                    wo2[1] = make_float2(link_bwd(lxm, A), xb);
                    wo2[2] = make_float2(link_fwd(ly.x, A), link_fwd(ly.y, A));
                    wo2[3] = make_float2(link_bwd(lyb.x, A), link_bwd(lyb.y, A));
                    wo2[4] = zf;
                    wo2[5] = zout;
                    sp = stay_weight2(wo2);
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        lwo0[k] = wo2[k].x;
                        lwo1[k] = wo2[k].y;
                    }
                    // for the next plane: the weights of its +z links from
                    // below; lane 0's left links are read two planes ahead
                    zin = zf;
                    zout = zb;
                    lxe = lxe1;
                    if (lane == 0 && ok_y && q + 2 < h.n)
                        lxe1 = left_link(z + 2);
                } else {
                    const WT* win = reinterpret_cast<const WT*>(ss);
                    sp = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(ss + SL.s) + os);
#pragma unroll
                    for (int k = 0; k < 6; ++k) win2[k] = lds_w2<WT>(win + k * C + os);
                }
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    q0.win[k] = win2[k].x;
                    q1.win[k] = win2[k].y;
                }
                // the populations of the sources, in pairs (.x for site 0, .y for site 1)
                const float2 rn2[6] = {make_float2(r_l, r_c.x), make_float2(r_c.y, r_r), r_u, r_d, br, r_a};
                q0.r[0] = r_l;   q0.r[1] = r_c.y; q0.r[2] = r_u.x; q0.r[3] = r_d.x; q0.r[4] = br.x; q0.r[5] = r_a.x;
                q1.r[0] = r_c.x; q1.r[1] = r_r;   q1.r[2] = r_u.y; q1.r[3] = r_d.y; q1.r[4] = br.y; q1.r[5] = r_a.y;
                q0.rc = r_c.x;
                q1.rc = r_c.y;
                float ro0, ro1;
                float2 mo0 = make_float2(0.f, 0.f), mo1 = make_float2(0.f, 0.f);
                float4 m_c = make_float4(0.f, 0.f, 0.f, 0.f);
                {
                    const float2 ro = pair_rho(win2, rn2, r_c, sp);
                    ro0 = ro.x;
                    ro1 = ro.y;
                }
                if constexpr (!RHO) {
                    const float2* mc = reinterpret_cast<const float2*>(sc + SL.m);
                    m_c = *reinterpret_cast<const float4*>(mc + o);
                    const float2 m_l = mc[o - 1], m_r = mc[o + 2];
                    const float4 m_u = *reinterpret_cast<const float4*>(mc + o - W);
                    const float4 m_d = *reinterpret_cast<const float4*>(mc + o + W);
                    const float4 m_a = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(sv + SL.m) + o);
                    const float4 Rp = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(ss + SL.R) + os);
                    q0.m[0] = m_l;                         q1.m[0] = make_float2(m_c.x, m_c.y);
                    q0.m[1] = make_float2(m_c.z, m_c.w);   q1.m[1] = m_r;
                    q0.m[2] = make_float2(m_u.x, m_u.y);   q1.m[2] = make_float2(m_u.z, m_u.w);
                    q0.m[3] = make_float2(m_d.x, m_d.y);   q1.m[3] = make_float2(m_d.z, m_d.w);
                    q0.m[4] = make_float2(bm.x, bm.y);     q1.m[4] = make_float2(bm.z, bm.w);
                    q0.m[5] = make_float2(m_a.x, m_a.y);   q1.m[5] = make_float2(m_a.z, m_a.w);
                    q0.mc = make_float2(m_c.x, m_c.y); q0.R = make_float2(Rp.x, Rp.y);
                    q1.mc = make_float2(m_c.z, m_c.w); q1.R = make_float2(Rp.z, Rp.w);
                    site_m(q0, sp.x, mo0);
                    site_m(q1, sp.y, mo1);
                }
                float muo0[3], muo1[3];
                float dd0[3] = {0.f, 0.f, 0.f}, dd1[3] = {0.f, 0.f, 0.f};
                int lab0 = 0, lab1 = 0;
                bool to_part = true;            // this plane's sums go to `part`
                if (REG) {
                    const unsigned int l2 = *reinterpret_cast<const unsigned short*>(ss + SL.lab + os);
                    lab0 = (int)(l2 & 0xffu);
                    lab1 = (int)(l2 >> 8);
                    // sites outside the lattice (ragged tiles) count for no region
                    const int labw = __shfl_sync(0xffffffffu, lab0, 0);
                    to_part = __all_sync(0xffffffffu, (!site0 || lab0 == labw) && (!site1 || lab1 == labw));
                    if (!to_part || labw != curlab) {
                        flush_run();
                        curlab = to_part ? labw : -1;
                    }
                }
#pragma unroll
                for (int n = 0; n < NMSD; ++n) {
                    const int a = axis_of[n];
                    const float* uc = reinterpret_cast<const float*>(sc + SL.mu[n]);
                    const float2 u_u = *reinterpret_cast<const float2*>(uc + o - W);
                    const float2 u_d = *reinterpret_cast<const float2*>(uc + o + W);
                    const float2 u_a = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sv + SL.mu[n]) + o);
                    const float nb0[6] = {uc[o - 1], muc[n].y, u_u.x, u_d.x, bmu[n].x, u_a.x};
                    const float nb1[6] = {muc[n].x, uc[o + 2], u_u.y, u_d.y, bmu[n].y, u_a.y};
                    const float2 nb2[6] = {make_float2(nb0[0], nb1[0]), make_float2(nb0[1], nb1[1]), u_u, u_d,
                                           bmu[n], u_a};
                    const float2 mo = pair_mu(win2, rn2, nb2, sp, muc[n], a);
                    muo0[n] = mo.x;
                    muo1[n] = mo.y;
                    if (LNK) {
                        dd0[n] = site_dmsd(lwo0, muc[n].x, q0.rc, a);
                        dd1[n] = site_dmsd(lwo1, muc[n].y, q1.rc, a);
                    } else if (dmx && n == 0) {
                        // x out-weights: w_+x(x) = win_+x(x + 1), w_-x(x) = win_-x(x - 1),
                        // from the lane's own pair and its neighbours' by shuffles; the
                        // tile's first column and last site from the tile-edge values
                        const float2 ex = lds_w2<WT>(reinterpret_cast<const WT*>(ss + SL.dx) + 2 * warp);
                        const float up = __shfl_up_sync(0xffffffffu, win2[1].y, 1);
                        const float dn = __shfl_down_sync(0xffffffffu, win2[0].x, 1);
                        const int last = min(kTX - 1, v.nx - 1 - tx * kTX);   // the tile's last site
                        const bool end0 = lane == (last >> 1) && !(last & 1);
                        const bool end1 = lane == (last >> 1) && (last & 1);
                        float wo0[6], wo1[6];
                        wo0[0] = end0 ? ex.y : win2[0].y;
                        wo0[1] = lane == 0 ? ex.x : up;
                        wo1[0] = end1 ? ex.y : dn;
                        wo1[1] = win2[1].x;
                        dd0[n] = site_dmsd(wo0, muc[n].x, q0.rc, 0);
                        dd1[n] = site_dmsd(wo1, muc[n].y, q1.rc, 0);
                    } else if (dmn >> n & 1) {
                        const float4 dm = lds_w4<WT>(reinterpret_cast<const WT*>(ss + SL.dm[n]) + 2 * os);
                        float wo0[6], wo1[6];
                        wo0[2 * a] = dm.x; wo0[2 * a + 1] = dm.y;
                        wo1[2 * a] = dm.z; wo1[2 * a + 1] = dm.w;
                        dd0[n] = site_dmsd(wo0, muc[n].x, q0.rc, a);
                        dd1[n] = site_dmsd(wo1, muc[n].y, q1.rc, a);
                    } else {
                        dd0[n] = site_dmsd_in(q0.win, q0.r, nb0, a);
                        dd1[n] = site_dmsd_in(q1.win, q1.r, nb1, a);
                    }
                    if (site0 && to_part) part[3 + a] += dd0[n];
                    if (site1 && to_part) part[3 + a] += dd1[n];
                }
                // both slots are read: release them before the stores
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&empty1[center]);
                    mbar_arrive(&empty2[sslot]);
                }
                // every site: its interior position (vector stores for a full
                // pair); pairs near a periodic face also write their ghost images
                {
                    const long long p = col + (long long)z * zplane;
                    if (site0 && site1) {
                        *reinterpret_cast<float2*>(v.rho_out + p) = make_float2(ro0, ro1);
                        if (!RHO) *reinterpret_cast<float4*>(v.m_out + p) = make_float4(mo0.x, mo0.y, mo1.x, mo1.y);
#pragma unroll
                        for (int n = 0; n < NMSD; ++n)
                            *reinterpret_cast<float2*>(v.mu_out[axis_of[n]] + p) = make_float2(muo0[n], muo1[n]);
                    } else if (site0) {
                        v.rho_out[p] = ro0;
                        if (!RHO) v.m_out[p] = mo0;
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) v.mu_out[axis_of[n]][p] = muo0[n];
                    }
                }
                if (images) {
                    const long long zoff = (long long)z * zplane;
                    if (site0) {
                        store_ghost_images(v.rho_out, v, x, y, zoff, ro0);
                        if (!RHO) store_ghost_images(v.m_out, v, x, y, zoff, mo0);
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) store_ghost_images(v.mu_out[axis_of[n]], v, x, y, zoff, muo0[n]);
                    }
                    if (site1) {
                        store_ghost_images(v.rho_out, v, x + 1, y, zoff, ro1);
                        if (!RHO) store_ghost_images(v.m_out, v, x + 1, y, zoff, mo1);
#pragma unroll
                        for (int n = 0; n < NMSD; ++n) store_ghost_images(v.mu_out[axis_of[n]], v, x + 1, y, zoff, muo1[n]);
                    }
                }
                if (site0 && to_part) { part[0] += mo0.x; part[1] += mo0.y; part[2] += ro0; }
                if (site1 && to_part) { part[0] += mo1.x; part[1] += mo1.y; part[2] += ro1; }
                if (REG && !to_part) {
                    touched |= __reduce_or_sync(0xffffffffu, (site0 ? 1u << lab0 : 0u) | (site1 ? 1u << lab1 : 0u));
#pragma unroll
                    for (int r = 0; r < (REG ? LPC_MAX_REGIONS : 1); ++r) {
                        const bool s0r = site0 && lab0 == r, s1r = site1 && lab1 == r;
                        preg[r][0] += (s0r ? mo0.x : 0.f) + (s1r ? mo1.x : 0.f);
                        preg[r][1] += (s0r ? mo0.y : 0.f) + (s1r ? mo1.y : 0.f);
                        preg[r][2] += (s0r ? ro0 : 0.f) + (s1r ? ro1 : 0.f);
#pragma unroll
                        for (int n = 0; n < NMSD; ++n)
                            preg[r][3 + n] += (s0r ? dd0[n] : 0.f) + (s1r ? dd1[n] : 0.f);
                    }
                }
                // this plane is the next one's "below"
                br = r_c;
                bm = m_c;
#pragma unroll
                for (int n = 0; n < NMSD; ++n) bmu[n] = muc[n];
                center = above;
            }
            if (!ok) break;
            // release the last plane of the item (loaded as the final "above")
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty1[center]);
            // item sums: a butterfly per warp; the last warp to finish the
            // item adds the warps in order and stores the item's FP64
            // partials (two buffers; a buffer is reused once its previous
            // item was combined, a bounded mbarrier wait)
            const int b = kitem & 1;
            const unsigned int use = kitem >> 1;
            if (use > 0) ok = mbar_wait_bounded(&ifree[b], (use - 1) & 1u);
            if (!ok) break;
            if (REG) {
                // close the run; the item's totals are the sums over regions
                flush_run();
                curlab = -1;
#pragma unroll
                for (int r = 0; r < (REG ? LPC_MAX_REGIONS : 1); ++r) {
                    part[0] += preg[r][0];
                    part[1] += preg[r][1];
                    part[2] += preg[r][2];
#pragma unroll
                    for (int n = 0; n < NMSD; ++n) part[3 + axis_of[n]] += preg[r][3 + n];
                }
            }
#pragma unroll
            for (int qq = 0; qq < kNumSums; ++qq) {
                const float t = warp_sum_f32(part[qq]);
                if (lane == 0) ired[(b * NC + warp) * KSP + qq] = (double)t;
                part[qq] = 0.f;
            }
            if (REG) {
                // only the regions this warp met in the item need a butterfly
#pragma unroll
                for (int r = 0; r < (REG ? LPC_MAX_REGIONS : 1); ++r) {
                    double* dst = ired + (b * NC + warp) * KSP + kNumSums * (1 + r);
                    if (touched >> r & 1u) {
#pragma unroll
                        for (int qq = 0; qq < 3; ++qq) {
                            const float t = warp_sum_f32(preg[r][qq]);
                            if (lane == 0) dst[qq] = (double)t;
                            preg[r][qq] = 0.f;
                        }
#pragma unroll
                        for (int a = 0, n = 0; a < 3; ++a) {
                            float t = 0.f;
                            if (MSD >> a & 1) {
                                t = warp_sum_f32(preg[r][3 + n]);
                                preg[r][3 + n] = 0.f;
                                ++n;
                            }
                            if (lane == 0) dst[3 + a] = (double)t;
                        }
                    } else if (lane < kNumSums) {
                        dst[lane] = 0.0;
                    }
                }
                touched = 0u;
            }
            __syncwarp();
            unsigned int last = 0u;
            if (lane == 0) {
                __threadfence_block();
                last = atomicAdd(&icount[b], 1u) == (unsigned)NC - 1u;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                if (lane < KS) {
                    double sum = 0.0;
                    for (int w = 0; w < NC; ++w) sum += ired[(b * NC + w) * KSP + lane];
                    const int item = ((h.za - v.zlo) / g.cz) * g.tiles + h.tile;
                    v.partials[(long long)item * KS + lane] = sum;
                }
                __syncwarp();
                if (lane == 0) {
                    icount[b] = 0u;
                    mbar_arrive(&ifree[b]);
                }
            }
            ++kitem;
        }
        if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            atomicExch(g.err, (unsigned int)LPC_ERR_TIMEOUT);
            // wait (bounded) until the copies of the last issued loads of both rings landed
            const unsigned int m1 = *issued1, m2 = *issued2;
            for (unsigned int l = m1 > (unsigned)S1 ? m1 - S1 : 0; l < m1; ++l)
                mbar_wait_bounded(&full1[l % S1], (l / S1) & 1u);
            for (unsigned int l = m2 > (unsigned)S2 ? m2 - S2 : 0; l < m2; ++l)
                mbar_wait_bounded(&full2[l % S2], (l / S2) & 1u);
        }
        __syncthreads();
        return;
    }
    // the rings are idle now: their memory is the final reduction's scratch
    if constexpr (REG)
        items_finish_regions<NC + 1, KS>(v, g.n_items, reinterpret_cast<double*>(ring1));
    else
        items_finish<NC + 1>(v, g.n_items, reinterpret_cast<double*>(ring1));
}

// ---------------------------------------------------------------------------
// Many lattices in one launch (serving): the work queue holds the items of
// every lattice of the launch, each lattice with its own tensor maps, view
// and item split (the split of its own launch), so a lattice's states and
// per-item sums are those of its own launch of k_step_tma1.  The warp that
// stores a lattice's last item (counted in the lattice's completion word)
// reduces that lattice's items with the arithmetic of its own launch's final
// reduction (items_reduce_warp), so its sums are bit for bit those of its own
// launch, and the reductions of different lattices overlap the remaining
// items instead of waiting for the end of the launch.  Lattices of one launch share the weight type,
// the tile height and the ghost width; the full step without moments, in
// the gather form (the form of the mid-size lattices that serving holds).

struct alignas(64) T1Lat {
    CUtensorMap rho, m, gwin, gs, gR;   // the lattice's current input buffer, gather form
    LatticeView v;
    int tiles_x, tiles, cz, n_items, item0;
};

struct T1MultiParams {
    T1Lat lat[kMaxMulti];
    int count, total_items;
    int W, S1, S2, slot1, slot2, tx1, tx2;
    unsigned int* work;                 // launch work queue (zeroed before the launch)
};
static_assert(sizeof(T1MultiParams) <= 32000, "kernel parameter space");

template <typename WT, int NC>
__global__ void __launch_bounds__((NC + 1) * 32, 1)
k_step_tma1_multi(const __grid_constant__ T1MultiParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (sa(smem_raw) & 127u)) & 127u);
    constexpr int TY = NC;
    constexpr int KSP = 8;
    const int W = P.W, S1 = P.S1, S2 = P.S2;
    const T1Slots SL = t1_slots(W, TY, 0, (int)sizeof(WT), false, false, 0, false, false);
    unsigned char* ring1 = smem;
    unsigned char* ring2 = smem + (size_t)S1 * P.slot1;
    uint64_t* full1 = reinterpret_cast<uint64_t*>(ring2 + (size_t)S2 * P.slot2);
    uint64_t* empty1 = full1 + S1;
    uint64_t* full2 = empty1 + S1;
    uint64_t* empty2 = full2 + S2;
    uint64_t* ifree = empty2 + S2;
    unsigned int* icount = reinterpret_cast<unsigned int*>(ifree + 2);
    SlotHdr* hdr = reinterpret_cast<SlotHdr*>(ifree + 3);
    double* ired = reinterpret_cast<double*>(hdr + S1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(ired + 2 * NC * KSP);
    volatile unsigned int* issued1 = reinterpret_cast<volatile unsigned int*>(abort_flag + 1);
    volatile unsigned int* issued2 = issued1 + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S1; ++s) {
            mbar_init(&full1[s], 1);
            mbar_init(&empty1[s], NC);
        }
        for (int s = 0; s < S2; ++s) {
            mbar_init(&full2[s], 1);
            mbar_init(&empty2[s], NC);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ifree[b], 1);
            icount[b] = 0u;
        }
        *abort_flag = 0;
        *issued1 = 0;
        *issued2 = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NC) {
        // ---------------- producer: one elected lane takes items of any lattice
        if (lane == 0) {
            for (int L = 0; L < P.count; ++L) {          // every lattice's descriptors
                prefetch_tmap(&P.lat[L].rho);
                prefetch_tmap(&P.lat[L].m);
                prefetch_tmap(&P.lat[L].gwin);
                prefetch_tmap(&P.lat[L].gs);
                prefetch_tmap(&P.lat[L].gR);
            }
            bool ok = true;
            Cursor c1{0, 0u}, c2{0, 0u};
            unsigned int n1 = 0, n2 = 0;
            auto state_load = [&](const T1Lat& T, int z, const SlotHdr& h, int bx, int by) -> bool {
                if (n1 >= (unsigned)S1 && !mbar_wait_bounded(&empty1[c1.slot], c1.ph ^ 1u)) return false;
                if (*abort_flag) return false;
                hdr[c1.slot] = h;
                unsigned char* st = ring1 + (size_t)c1.slot * P.slot1;
                uint64_t* fb = &full1[c1.slot];
                fence_proxy_async();
                if (h.tile < 0) {
                    mbar_arrive(fb);
                } else {
                    mbar_expect_tx(fb, (uint32_t)P.tx1);
                    tma3(st, &T.rho, fb, bx, by, z);
                    tma3(st + SL.m, &T.m, fb, 2 * bx, by, z);
                }
                *issued1 = ++n1;
                c1.next(S1);
                return true;
            };
            for (;;) {
                const int item = (int)atomicAdd(P.work, 1u);
                if (item >= P.total_items) break;
                int L = 0;
                while (L + 1 < P.count && item >= P.lat[L + 1].item0) ++L;
                const T1Lat& T = P.lat[L];
                const int local = item - T.item0;
                const int nz = T.v.nz;
                const int tile = local % T.tiles;
                const int za = T.v.zlo + (local / T.tiles) * T.cz;
                const int n = min(T.cz, T.v.zhi - za);
                const int tx = tile % T.tiles_x, ty = tile / T.tiles_x;
                const int bx = tx * kTX;
                const int by = ty * TY + T.v.G - 1;
                const int sx = tx * kTX, sy = ty * TY;
                const SlotHdr h{tile, za, n, L};
                ok = state_load(T, za == 0 ? nz - 1 : za - 1, h, bx, by) && state_load(T, za, h, bx, by);
                for (int q = 0; q < n && ok; ++q) {
                    if (n2 >= (unsigned)S2) ok = mbar_wait_bounded(&empty2[c2.slot], c2.ph ^ 1u);
                    if (!ok || *abort_flag) { ok = false; break; }
                    {
                        unsigned char* st = ring2 + (size_t)c2.slot * P.slot2;
                        uint64_t* fb = &full2[c2.slot];
                        const int z = za + q;
                        fence_proxy_async();
                        mbar_expect_tx(fb, (uint32_t)P.tx2);
                        tma4(st, &T.gwin, fb, sx, sy, z, 0);
                        tma3(st + SL.s, &T.gs, fb, sx, sy, z);
                        tma3(st + SL.R, &T.gR, fb, 2 * sx, sy, z);
                        *issued2 = ++n2;
                        c2.next(S2);
                    }
                    const int za1 = za + q + 1;
                    ok = state_load(T, za1 == nz ? 0 : za1, h, bx, by);
                }
                if (!ok) break;
            }
            if (ok) ok = state_load(P.lat[0], 0, SlotHdr{-1, 0, 0, 0}, 0, 0);
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---------------- consumer warps: core row `warp`, sites x0 + 2 lane + {0, 1}
        float part[3] = {0.f, 0.f, 0.f};
        bool ok = true;
        Cursor w1{0, 0u}, w2{0, 0u};
        unsigned int kitem = 0;
        const int o = (warp + 1) * W + P.lat[0].v.G + 2 * lane;   // one ghost width for the launch
        const int os = warp * kTX + 2 * lane;
        const int C = TY * kTX;
        for (;;) {
            ok = mbar_wait_bounded(&full1[w1.slot], w1.ph);
            if (!ok) break;
            const SlotHdr h = hdr[w1.slot];
            if (h.tile < 0) break;
            const T1Lat& T = P.lat[h.pad];
            const LatticeView& v = T.v;
            const int G = v.G;
            const int tx = h.tile % T.tiles_x, ty = h.tile / T.tiles_x;
            const int x = tx * kTX + 2 * lane;
            const int y = ty * TY + warp;
            const bool ok_y = y < v.ny;
            const bool site0 = ok_y && x < v.nx;
            const bool site1 = ok_y && x + 1 < v.nx;
            const bool images = (v.per_x && (x < G || x + 1 >= v.nx - G)) || (v.per_y && (y < G || y >= v.ny - G));
            const long long col = (long long)(y + G) * v.Xp + (x + G);
            const long long zplane = (long long)v.Xp * v.Yp;
            float* rho_out = v.rho_out;
            float2* m_out = v.m_out;
            float2 br;
            float4 bm;
            {
                const unsigned char* s0 = ring1 + (size_t)w1.slot * P.slot1;
                br = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(s0) + o);
                bm = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(s0 + SL.m) + o);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty1[w1.slot]);
                w1.next(S1);
            }
            ok = mbar_wait_bounded(&full1[w1.slot], w1.ph);
            int center = w1.slot;
            w1.next(S1);
            for (int q = 0; q < h.n && ok; ++q) {
                const int z = h.za + q;
                const int sslot = w2.slot;
                ok = mbar_wait_bounded(&full2[sslot], w2.ph);
                w2.next(S2);
                const int above = w1.slot;
                ok = ok && mbar_wait_bounded(&full1[above], w1.ph);
                w1.next(S1);
                if (!ok || *abort_flag) { ok = false; break; }
                const unsigned char* sc = ring1 + (size_t)center * P.slot1;
                const unsigned char* sv = ring1 + (size_t)above * P.slot1;
                const unsigned char* ss = ring2 + (size_t)sslot * P.slot2;
                const float* rc = reinterpret_cast<const float*>(sc);
                const float2 r_c = *reinterpret_cast<const float2*>(rc + o);
                const float r_l = rc[o - 1], r_r = rc[o + 2];
                const float2 r_u = *reinterpret_cast<const float2*>(rc + o - W);
                const float2 r_d = *reinterpret_cast<const float2*>(rc + o + W);
                const float2 r_a = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(sv) + o);
                const WT* win = reinterpret_cast<const WT*>(ss);
                const float2 sp = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(ss + SL.s) + os);
                float2 win2[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) win2[k] = lds_w2<WT>(win + k * C + os);
                SiteIn q0, q1;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    q0.win[k] = win2[k].x;
                    q1.win[k] = win2[k].y;
                }
                const float2 rn2[6] = {make_float2(r_l, r_c.x), make_float2(r_c.y, r_r), r_u, r_d, br, r_a};
                const float2 ro = pair_rho(win2, rn2, r_c, sp);
                const float2* mc = reinterpret_cast<const float2*>(sc + SL.m);
                const float4 m_c = *reinterpret_cast<const float4*>(mc + o);
                const float2 m_l = mc[o - 1], m_r = mc[o + 2];
                const float4 m_u = *reinterpret_cast<const float4*>(mc + o - W);
                const float4 m_d = *reinterpret_cast<const float4*>(mc + o + W);
                const float4 m_a = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(sv + SL.m) + o);
                const float4 Rp = *reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(ss + SL.R) + os);
                q0.m[0] = m_l;                         q1.m[0] = make_float2(m_c.x, m_c.y);
                q0.m[1] = make_float2(m_c.z, m_c.w);   q1.m[1] = m_r;
                q0.m[2] = make_float2(m_u.x, m_u.y);   q1.m[2] = make_float2(m_u.z, m_u.w);
                q0.m[3] = make_float2(m_d.x, m_d.y);   q1.m[3] = make_float2(m_d.z, m_d.w);
                q0.m[4] = make_float2(bm.x, bm.y);     q1.m[4] = make_float2(bm.z, bm.w);
                q0.m[5] = make_float2(m_a.x, m_a.y);   q1.m[5] = make_float2(m_a.z, m_a.w);
                q0.mc = make_float2(m_c.x, m_c.y); q0.R = make_float2(Rp.x, Rp.y);
                q1.mc = make_float2(m_c.z, m_c.w); q1.R = make_float2(Rp.z, Rp.w);
                float2 mo0, mo1;
                site_m(q0, sp.x, mo0);
                site_m(q1, sp.y, mo1);
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&empty1[center]);
                    mbar_arrive(&empty2[sslot]);
                }
                {
                    const long long p = col + (long long)z * zplane;
                    if (site0 && site1) {
                        *reinterpret_cast<float2*>(rho_out + p) = ro;
                        *reinterpret_cast<float4*>(m_out + p) = make_float4(mo0.x, mo0.y, mo1.x, mo1.y);
                    } else if (site0) {
                        rho_out[p] = ro.x;
                        m_out[p] = mo0;
                    }
                }
                if (images) {
                    const long long zoff = (long long)z * zplane;
                    if (site0) {
                        store_ghost_images(rho_out, v, x, y, zoff, ro.x);
                        store_ghost_images(m_out, v, x, y, zoff, mo0);
                    }
                    if (site1) {
                        store_ghost_images(rho_out, v, x + 1, y, zoff, ro.y);
                        store_ghost_images(m_out, v, x + 1, y, zoff, mo1);
                    }
                }
                if (site0) { part[0] += mo0.x; part[1] += mo0.y; part[2] += ro.x; }
                if (site1) { part[0] += mo1.x; part[1] += mo1.y; part[2] += ro.y; }
                br = r_c;
                bm = m_c;
                center = above;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty1[center]);
            const int b = kitem & 1;
            const unsigned int use = kitem >> 1;
            if (use > 0) ok = mbar_wait_bounded(&ifree[b], (use - 1) & 1u);
            if (!ok) break;
            // the item's sums, as in k_step_tma1: a butterfly per warp, the
            // last warp of the item adds the warps in order
#pragma unroll
            for (int qq = 0; qq < kNumSums; ++qq) {
                const float t = warp_sum_f32(qq < 3 ? part[qq] : 0.f);
                if (lane == 0) ired[(b * NC + warp) * KSP + qq] = (double)t;
                if (qq < 3) part[qq] = 0.f;
            }
            __syncwarp();
            unsigned int last = 0u;
            if (lane == 0) {
                __threadfence_block();
                last = atomicAdd(&icount[b], 1u) == (unsigned)NC - 1u;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                if (lane < kNumSums) {
                    double sum = 0.0;
                    for (int w = 0; w < NC; ++w) sum += ired[(b * NC + w) * KSP + lane];
                    const int item = ((h.za - v.zlo) / T.cz) * T.tiles + h.tile;
                    v.partials[(long long)item * kNumSums + lane] = sum;
                    __threadfence();
                }
                __syncwarp();
                unsigned int done_items = 0u;
                if (lane == 0) {
                    icount[b] = 0u;
                    mbar_arrive(&ifree[b]);
                    done_items = atomicAdd(v.counter, 1u);     // the lattice's items stored so far
                }
                done_items = __shfl_sync(0xffffffffu, done_items, 0);
                if (done_items == (unsigned)T.n_items - 1u) {
                    // the lattice's last item: this warp reduces its items, in
                    // the fixed order of the lattice's own launch
                    __threadfence();
                    items_reduce_warp<NC + 1>(v, T.n_items);
                    if (lane == 0) *v.counter = 0u;
                }
            }
            ++kitem;
        }
        if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            for (int L = 0; L < P.count; ++L) atomicExch(P.lat[L].v.counter + 1, (unsigned int)LPC_ERR_TIMEOUT);
            const unsigned int m1 = *issued1, m2 = *issued2;
            for (unsigned int l = m1 > (unsigned)S1 ? m1 - S1 : 0; l < m1; ++l)
                mbar_wait_bounded(&full1[l % S1], (l / S1) & 1u);
            for (unsigned int l = m2 > (unsigned)S2 ? m2 - S2 : 0; l < m2; ++l)
                mbar_wait_bounded(&full2[l % S2], (l / S2) & 1u);
        }
        __syncthreads();
        return;
    }
}

template <typename WT, int NC>
void* t1_multi_fn() { return reinterpret_cast<void*>(&k_step_tma1_multi<WT, NC>); }

void* t1_multi_kernel(int TY, int wdtype) {
    const bool bf = wdtype == LPC_WEIGHTS_BF16;
    if (TY == 16) return bf ? t1_multi_fn<__nv_bfloat16, 16>() : t1_multi_fn<float, 16>();
    if (TY == 12) return bf ? t1_multi_fn<__nv_bfloat16, 12>() : t1_multi_fn<float, 12>();
    return bf ? t1_multi_fn<__nv_bfloat16, 8>() : t1_multi_fn<float, 8>();
}

template <typename WT, int MSD, int NC, bool REG, bool LNK>
void* t1_fn() { return reinterpret_cast<void*>(&k_step_tma1<WT, MSD, NC, false, REG, LNK>); }

template <int NC, bool LNK>
void* t1_rho_kernel(int wdtype) {
    return wdtype == LPC_WEIGHTS_BF16 ? reinterpret_cast<void*>(&k_step_tma1<__nv_bfloat16, 0, NC, true, false, LNK>)
                                      : reinterpret_cast<void*>(&k_step_tma1<float, 0, NC, true, false, LNK>);
}

template <int NC, bool REG, bool LNK>
void* t1_kernel_shape(int wdtype, int msd) {
    static void* tab[2][8] = {
        {t1_fn<float, 0, NC, REG, LNK>(), t1_fn<float, 1, NC, REG, LNK>(), t1_fn<float, 2, NC, REG, LNK>(),
         t1_fn<float, 3, NC, REG, LNK>(), t1_fn<float, 4, NC, REG, LNK>(), t1_fn<float, 5, NC, REG, LNK>(),
         t1_fn<float, 6, NC, REG, LNK>(), t1_fn<float, 7, NC, REG, LNK>()},
        {t1_fn<__nv_bfloat16, 0, NC, REG, LNK>(), t1_fn<__nv_bfloat16, 1, NC, REG, LNK>(),
         t1_fn<__nv_bfloat16, 2, NC, REG, LNK>(), t1_fn<__nv_bfloat16, 3, NC, REG, LNK>(),
         t1_fn<__nv_bfloat16, 4, NC, REG, LNK>(), t1_fn<__nv_bfloat16, 5, NC, REG, LNK>(),
         t1_fn<__nv_bfloat16, 6, NC, REG, LNK>(), t1_fn<__nv_bfloat16, 7, NC, REG, LNK>()}};
    return tab[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
}

// Tile heights (= consumer warps) tried in order; the first whose rings keep
// at least LPC_T1_MIN_DEPTH planes in flight is used (the last one always).
constexpr int kShapes[3] = {16, 12, 8};

struct T1Choice {
    int TY, W, S1, S2, depth;
    T1Slots L;
    int smem;
};

// Box width of the state: the 64 core columns plus G on each side, rounded
// up to 16 bytes.
int t1_box_width(int G) { return (kTX + 2 * G + 3) / 4 * 4; }

// Ring depth d and shared memory of a tile height: S1 = d + 2 state slots
// (centre and above held), S2 = d + 1 static slots (centre held); per slot one
// full and one empty barrier, and a header per state slot.
void t1_rings(T1Choice& c, int TY, int nmsd, int wb, bool rho_only, bool reg, int dmn, bool dmx, bool lnk) {
    const T1Slots L = t1_slots(c.W, TY, nmsd, wb, rho_only, reg, dmn, dmx, lnk);
    const int ksp = reg ? ItemSums<true>::KSP : ItemSums<false>::KSP;
    const int fixed = 128 + 3 * 8 + 2 * TY * ksp * 8 + 64;   // slack, item barriers/counts/sums, flags
    const int budget = device_props().max_smem_optin - 1024 - fixed;
    const int per1 = L.bytes1 + 16 + 16, per2 = L.bytes2 + 16;
    int d = (budget - 2 * per1 - per2) / (per1 + per2);
    if (d > 8) d = 8;
    c.TY = TY;
    c.depth = d;
    c.S1 = d + 2;
    c.S2 = d + 1;
    c.L = L;
    c.smem = fixed + c.S1 * per1 + c.S2 * per2;
}

// The tile height comes from the full step without regions (so that one set
// of tensor maps serves every mode); the rho-only step and the step with
// region sums re-size their rings for it.
T1Choice t1_choose(const LatticeView& v, int wdtype, bool rho_only = false, bool reg = false) {
    const int nmsd = popc(v.msd_axes);
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    const bool lnk = v.lnk != nullptr;         // the lattice's static data is in link form
    // pairs staged where the lattice keeps them (source-attributed MSD sums)
    const int dmn = t1_dm_staged(v.msd_axes, !lnk && v.gdm);
    const bool dmx = !lnk && v.gdm && (v.msd_axes & 1);
    T1Choice c{};
    c.W = t1_box_width(v.G);
    bool chosen = false;
    if (v.t1_ty == 8 || v.t1_ty == 12 || v.t1_ty == 16) {       // set by the caller or the autotuner
        t1_rings(c, v.t1_ty, nmsd, wb, false, false, dmn, dmx, lnk);
        chosen = c.depth >= 1;
    }
    for (int i = 0; i < 3 && !chosen; ++i) {
        t1_rings(c, kShapes[i], nmsd, wb, false, false, dmn, dmx, lnk);
        if ((c.depth >= LPC_T1_MIN_DEPTH && v.ny > kShapes[i] / 2) || i == 2) break;
    }
    if (rho_only) t1_rings(c, c.TY, 0, wb, true, false, 0, false, lnk);
    else if (reg) t1_rings(c, c.TY, nmsd, wb, false, true, t1_dm_staged(v.msd_axes, !lnk), !lnk && (v.msd_axes & 1), lnk);
    return c;
}

void* t1_kernel(int TY, int wdtype, int msd, bool rho_only = false, bool reg = false, bool lnk = false) {
    if (rho_only) {
        if (lnk) return TY == 16 ? t1_rho_kernel<16, true>(wdtype)
                                 : (TY == 12 ? t1_rho_kernel<12, true>(wdtype) : t1_rho_kernel<8, true>(wdtype));
        return TY == 16 ? t1_rho_kernel<16, false>(wdtype)
                        : (TY == 12 ? t1_rho_kernel<12, false>(wdtype) : t1_rho_kernel<8, false>(wdtype));
    }
    if (reg && lnk) {
        if (TY == 16) return t1_kernel_shape<16, true, true>(wdtype, msd);
        if (TY == 12) return t1_kernel_shape<12, true, true>(wdtype, msd);
        return t1_kernel_shape<8, true, true>(wdtype, msd);
    }
    if (reg) {
        if (TY == 16) return t1_kernel_shape<16, true, false>(wdtype, msd);
        if (TY == 12) return t1_kernel_shape<12, true, false>(wdtype, msd);
        return t1_kernel_shape<8, true, false>(wdtype, msd);
    }
    if (lnk) {
        if (TY == 16) return t1_kernel_shape<16, false, true>(wdtype, msd);
        if (TY == 12) return t1_kernel_shape<12, false, true>(wdtype, msd);
        return t1_kernel_shape<8, false, true>(wdtype, msd);
    }
    if (TY == 16) return t1_kernel_shape<16, false, false>(wdtype, msd);
    if (TY == 12) return t1_kernel_shape<12, false, false>(wdtype, msd);
    return t1_kernel_shape<8, false, false>(wdtype, msd);
}

}  // namespace

cudaError_t t1_prepare(int wdtype, int msd) {
    static bool done[2][8] = {};
    bool& d = done[wdtype == LPC_WEIGHTS_BF16][msd & 7];
    if (d) return cudaSuccess;
    // per tile height: full step, rho-only step, with regions, link form, link-form rho-only step,
    // link form with regions
    for (int i = 0; i < 18; ++i) {
        const int mode = i / 3;
        void* fn = t1_kernel(kShapes[i % 3], wdtype, msd, mode == 1 || mode == 4, mode == 2 || mode == 5, mode >= 3);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 device_props().max_smem_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    d = true;
    return cudaSuccess;
}

// Item partials fit the lattice's partials buffer (sm_count * 32 * kMaxTB
// entries of kNumSums doubles).
static int t1_max_items() { return device_props().sm_count * 32 * kMaxTB; }

// The fused region sums need labels of width 64 per tile row, ring memory for
// the final reduction's scratch (32 doubles per warp) and a ring depth of at
// least one plane.
bool t1_fused_regions(const LatticeView& v, int wdtype) {
    if (v.nreg <= 0 || !v.region) return false;
    const T1Choice c = t1_choose(v, wdtype, false, true);
    const long long scratch = 32LL * (c.TY + 1) * 8;
    const long long rings = (long long)c.S1 * c.L.bytes1 + (long long)c.S2 * c.L.bytes2;
    return c.depth >= 1 && scratch <= rings && v.Xr == v.Xs;
}

int t1_tile_rows(const LatticeView& v, int wdtype) { return t1_choose(v, wdtype).TY; }

int t1_default_items_per_cta() { return LPC_T1_ITEMS_PER_CTA; }

// Work items of one lattice at tile height TY: tiles of 64 x TY sites, the
// tile index fastest, over z-chunks of cz planes of [zlo, zhi); about
// items_per_cta items per CTA of a one-CTA-per-SM grid, chunks of at least 8
// planes (the multi-lattice launch uses the same split, so a lattice's
// per-item sums are the same in either launch).
void t1_items(const LatticeView& v, int TY, int* tiles_x, int* tiles, int* cz_out, int* n_items) {
    *tiles_x = (v.nx + kTX - 1) / kTX;
    *tiles = *tiles_x * ((v.ny + TY - 1) / TY);
    const int sms = device_props().sm_count;
    const int nzu = v.zhi - v.zlo;              // planes updated
    const long long ipc = v.t1_ipc > 0 ? v.t1_ipc : LPC_T1_ITEMS_PER_CTA;
    long long cz = (long long)*tiles * nzu / (ipc * sms);
    if (cz < 8) cz = 8;
    if (cz > nzu) cz = nzu;
    while ((long long)*tiles * ((nzu + cz - 1) / cz) > t1_max_items() && cz < nzu) cz *= 2;
    if (cz > nzu) cz = nzu;
    *cz_out = (int)cz;
    *n_items = *tiles * ((nzu + *cz_out - 1) / *cz_out);
}

bool t1_supported(const LatticeView& v, int wdtype) {
    const T1Choice c = t1_choose(v, wdtype);
    const long long tiles = (long long)((v.nx + kTX - 1) / kTX) * ((v.ny + c.TY - 1) / c.TY);
    return v.G >= 2 && v.G % 2 == 0 && encode_fn() != nullptr && c.depth >= 1 && tiles <= t1_max_items();
}

bool t1_encode_maps(const LatticeView& v, int wdtype, TBMaps* maps) {
    if (!v.gwin && !v.lnk) return false;
    const T1Choice c = t1_choose(v, wdtype);
    const cuuint64_t Xp = (cuuint64_t)v.Xp, Yp = (cuuint64_t)v.Yp, nz = (cuuint64_t)v.nz;
    const cuuint32_t W = (cuuint32_t)c.W, TY = (cuuint32_t)c.TY;
    bool ok = true;
    {
        const cuuint64_t dims[3] = {Xp, Yp, nz};
        const cuuint64_t str[2] = {Xp * 4, Xp * Yp * 4};
        const cuuint32_t box[3] = {W, TY + 2, 1};
        ok = ok && tma_encode(&maps->rho, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.rho_in, dims, str, box);
        for (int a = 0, n = 0; a < 3; ++a)
            if (v.msd_axes >> a & 1)
                ok = ok && tma_encode(&maps->mu[n++], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.mu_in[a], dims, str, box);
    }
    {
        const cuuint64_t dims[3] = {2 * Xp, Yp, nz};
        const cuuint64_t str[2] = {Xp * 8, Xp * Yp * 8};
        const cuuint32_t box[3] = {2 * W, TY + 2, 1};
        ok = ok && tma_encode(&maps->m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.m_in, dims, str, box);
    }
    {
        const cuuint64_t Xs = (cuuint64_t)v.Xs, ny = (cuuint64_t)v.ny;
        const cuuint64_t e = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
        const CUtensorMapDataType dt =
            wdtype == LPC_WEIGHTS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        if (v.lnk) {
            // link planes [3][nz][ny + 1][Xs]: boxes of TY rows (x and z links)
            // and TY + 1 rows (y links, with the row above)
            const cuuint64_t ny1 = (cuuint64_t)v.ny1;
            const cuuint64_t dl[4] = {Xs, ny1, nz, 3};
            const cuuint64_t sl[3] = {Xs * e, Xs * ny1 * e, Xs * ny1 * nz * e};
            const cuuint32_t bl1[4] = {(cuuint32_t)kTX, TY, 1, 1};
            const cuuint32_t bl2[4] = {(cuuint32_t)kTX, TY + 1, 1, 1};
            ok = ok && tma_encode(&maps->glnk1, dt, 4, v.lnk, dl, sl, bl1);
            ok = ok && tma_encode(&maps->glnk2, dt, 4, v.lnk, dl, sl, bl2);
        } else {
            const cuuint64_t dw[4] = {Xs, ny, nz, 6};
            const cuuint64_t sw[3] = {Xs * e, Xs * ny * e, Xs * ny * nz * e};
            const cuuint32_t bw[4] = {(cuuint32_t)kTX, TY, 1, 6};
            ok = ok && tma_encode(&maps->gwin, dt, 4, v.gwin, dw, sw, bw);
            const cuuint64_t ds[3] = {Xs, ny, nz};
            const cuuint64_t ss[2] = {Xs * 4, Xs * ny * 4};
            const cuuint32_t bs[3] = {(cuuint32_t)kTX, TY, 1};
            ok = ok && tma_encode(&maps->gs, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.gs, ds, ss, bs);
        }
        const cuuint64_t dr[3] = {2 * Xs, ny, nz};
        const cuuint64_t sr[2] = {Xs * 8, Xs * ny * 8};
        const cuuint32_t br[3] = {(cuuint32_t)(2 * kTX), TY, 1};
        ok = ok && tma_encode(&maps->gR, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, v.gR, dr, sr, br);
        if (v.gdm) {
            const cuuint64_t dd[4] = {2 * Xs, ny, nz, 3};
            const cuuint64_t sd[3] = {Xs * 2 * e, Xs * ny * 2 * e, Xs * ny * nz * 2 * e};
            const cuuint32_t bd[4] = {(cuuint32_t)(2 * kTX), TY, 1, 1};
            ok = ok && tma_encode(&maps->gdm, dt, 4, v.gdm, dd, sd, bd);
        }
        if (v.gdx) {
            // tile-edge x out-weights [nz][tiles_x][nyp][2]: a box of the TY rows of one tile
            const cuuint64_t nyp = (cuuint64_t)((v.ny + 7) / 8 * 8), ntx = (cuuint64_t)((v.nx + kTX - 1) / kTX);
            const cuuint64_t dx[3] = {2 * nyp, ntx, nz};
            const cuuint64_t sx[2] = {2 * nyp * e, 2 * nyp * ntx * e};
            const cuuint32_t bx[3] = {2 * TY, 1, 1};
            ok = ok && tma_encode(&maps->gdx, dt, 3, v.gdx, dx, sx, bx);
        }
        if (v.region && v.Xr == v.Xs) {
            const cuuint64_t dl[3] = {Xs, ny, nz};
            const cuuint64_t sl[2] = {Xs, Xs * ny};
            const cuuint32_t bl[3] = {(cuuint32_t)kTX, TY, 1};
            ok = ok && tma_encode(&maps->glab, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, v.region, dl, sl, bl);
        }
    }
    return ok;
}

// A lattice joins a multi-lattice launch when it runs the TMA-fed one-step
// kernel from the gather form, without moments, regions or halo planes.
bool t1_multi_member(const LatticeView& v, int wdtype) {
    return v.gwin && !v.lnk && !v.gdm && v.msd_axes == 0 && v.nreg == 0 && v.zlo == 0 && v.zhi == v.nz &&
           t1_supported(v, wdtype);
}

int t1_multi_group(const LatticeView& v, int wdtype) {
    return (t1_choose(v, wdtype).TY * 16 + v.G) * 2 + (wdtype == LPC_WEIGHTS_BF16 ? 1 : 0);
}

cudaError_t launch_tma1_multi(const LatticeView* views, const TBMaps* const* maps, int count, int wdtype,
                              unsigned int* words, cudaStream_t st) {
    if (count < 1 || count > kMaxMulti) return cudaErrorInvalidValue;
    static thread_local T1MultiParams P;
    const T1Choice c = t1_choose(views[0], wdtype);
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    P.W = c.W;
    P.S1 = c.S1;
    P.S2 = c.S2;
    P.slot1 = c.L.bytes1;
    P.slot2 = c.L.bytes2;
    P.tx1 = (c.TY + 2) * c.W * 12;
    P.tx2 = c.TY * kTX * (6 * wb + 4 + 8);
    int total = 0;
    for (int i = 0; i < count; ++i) {
        const LatticeView& v = views[i];
        if (!t1_multi_member(v, wdtype) || t1_multi_group(v, wdtype) != t1_multi_group(views[0], wdtype))
            return cudaErrorInvalidValue;
        T1Lat& T = P.lat[i];
        T.rho = maps[i]->rho;
        T.m = maps[i]->m;
        T.gwin = maps[i]->gwin;
        T.gs = maps[i]->gs;
        T.gR = maps[i]->gR;
        T.v = v;
        t1_items(v, c.TY, &T.tiles_x, &T.tiles, &T.cz, &T.n_items);
        if (T.n_items > t1_max_items()) return cudaErrorInvalidConfiguration;
        T.item0 = total;
        total += T.n_items;
    }
    P.count = count;
    P.total_items = total;
    P.work = words;
    static bool attr_done[2][3] = {};
    bool& ad = attr_done[wb == 2][c.TY == 16 ? 0 : (c.TY == 12 ? 1 : 2)];
    void* fn = t1_multi_kernel(c.TY, wdtype);
    if (!ad) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 device_props().max_smem_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        ad = true;
    }
    cudaError_t e = cudaMemsetAsync(words, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int grid = device_props().sm_count;
    if (grid > total) grid = total;
    void* args[] = {&P};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((c.TY + 1) * 32), args, (size_t)c.smem, st);
}

cudaError_t launch_tma1(const LatticeView& v, int wdtype, const TBMaps& maps, unsigned int* err,
                        cudaStream_t st, bool rho_only) {
    if (!v.gwin && !v.lnk) return cudaErrorInvalidValue;
    const bool lnk = v.lnk != nullptr;
    const bool reg = !rho_only && t1_fused_regions(v, wdtype);
    const T1Choice c = t1_choose(v, wdtype, rho_only, reg);
    const int nmsd = rho_only ? 0 : popc(v.msd_axes);
    const int wb = wdtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    T1Geom g;
    g.W = c.W;
    g.TY = c.TY;
    g.S1 = c.S1;
    g.S2 = c.S2;
    g.slot1 = c.L.bytes1;
    g.slot2 = c.L.bytes2;
    g.tx1 = (c.TY + 2) * c.W * (rho_only ? 4 : 12 + 4 * nmsd);
    g.dm_src = (!rho_only && !lnk && v.gdm) ? 1 : 0;
    const int dmn = t1_dm_staged(v.msd_axes & (rho_only ? 0 : 7), !rho_only && !lnk && (reg || g.dm_src));
    const bool dmx = !rho_only && !lnk && (reg || g.dm_src) && (v.msd_axes & 1);
    g.abig = v.link_a;
    if (lnk)   // three link boxes (one with the row above), R and the labels
        g.tx2 = c.TY * kTX * (3 * wb + (rho_only ? 0 : 8) + (reg ? 1 : 0)) + kTX * wb;
    else
        g.tx2 = c.TY * kTX * (6 * wb + 4 + (rho_only ? 0 : 8 + 2 * wb * popc(dmn)) + (reg ? 1 : 0)) +
                (dmx ? c.TY * 2 * wb : 0);
    t1_items(v, c.TY, &g.tiles_x, &g.tiles, &g.cz, &g.n_items);
    const int sms = device_props().sm_count;
    if (g.n_items > t1_max_items()) return cudaErrorInvalidConfiguration;
    g.err = err;
    g.work = err + 7;
    cudaError_t e = t1_prepare(wdtype, v.msd_axes);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(g.work, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int grid = sms;
    if (grid > g.n_items) grid = g.n_items;
    LatticeView vv = v;
    TBMaps mm = maps;
    void* args[] = {&mm, &vv, &g};
    return cudaLaunchKernel(t1_kernel(c.TY, wdtype, v.msd_axes, rho_only, reg, lnk), dim3((unsigned)grid),
                            dim3((c.TY + 1) * 32), args, (size_t)c.smem, st);
}

}  // namespace lpc
