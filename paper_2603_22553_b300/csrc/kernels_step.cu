// One time step per launch (the "step1" schedule) and its batched form.
//
// A block of 32 x 8 threads owns a 32 x 8 tile of (x, y) columns (one site
// per thread, a warp per row) and walks a chunk of z planes.  Each thread
// keeps the state and out-weights of the planes below, at and above its
// site in registers and prefetches ahead: the state and -z weight of the
// plane two above, the remaining weights and R of the plane above (register
// sets rotate through a 4-way unrolled loop, so no moves).  x neighbours come
// from the neighbouring lanes by shuffles (the row's end lanes prefetch the
// column just outside the row); y neighbours are read from L1 (rows of the
// same block) or L2.  All offsets are 32-bit (padded lattices hold fewer
// than 2^31 sites), so a load costs one address operation.  HBM traffic is
// one read of state, weights and R per site and one write of the state.
//
// Blocks loop over (x-tile, y-tile, z-chunk) work items.  Each thread sums
// its sites of an item in FP32; one warp butterfly per item turns thread
// sums into FP64 per-warp sums; blocks combine in FP64 and the last block
// writes the step's M, P and dMSD into the device history.
#include "lpc_internal.cuh"

namespace lpc {

namespace {

constexpr int BX = 32, BY = 8;             // threads per block: lanes x rows
constexpr int TX = BX, TY = BY;            // tile 32 x 8 sites
constexpr int NWARP = BY;

// Per-array base pointers of one launch (weights as 6 plane pointers).
template <typename WT>
struct Ptrs {
    const float* rho;
    const float2* m;
    const float* mu[3];
    const WT* w[6];
    const float2* R;
};

template <typename WT>
__device__ __forceinline__ Ptrs<WT> make_ptrs(const LatticeView& v) {
    Ptrs<WT> P;
    P.rho = v.rho_in;
    P.m = v.m_in;
    for (int a = 0; a < 3; ++a) P.mu[a] = v.mu_in[a];
    const WT* W = static_cast<const WT*>(v.w);
    for (int k = 0; k < 6; ++k) P.w[k] = W + (long long)k * v.Np;
    P.R = v.R;
    return P;
}

// One plane of a thread's column (and, for the row's end lanes, of the column
// just outside the row: h*).
template <int MSD>
struct Pl {
    float r;
    float2 m;
    float w[6];
    float mu[3];
    float hr, hw;
    float2 hm;
    float hmu[3];
};

struct Col {
    int o;                    // padded offset of the site in its plane
    int lane, x, y;
    bool load, site;          // thread loads; the site is a lattice site
    int halo;                 // -1: lane 0 loads x-1, +1: lane 31 loads x+1, 0: none
};

// early part: state, -z out-weight, end lanes' outside column
template <typename WT, int MSD>
__device__ __forceinline__ void load_early(Pl<MSD>& P, const Ptrs<WT>& A, int zo, const Col& c) {
    if (!c.load) return;
    const int i = zo + c.o;
    P.r = __ldg(A.rho + i);
    P.m = __ldg(A.m + i);
    P.w[5] = ldw<WT>(A.w[5] + i);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (MSD >> a & 1) P.mu[a] = __ldg(A.mu[a] + i);
    if (c.halo != 0) {
        const int j = i + c.halo;
        P.hr = __ldg(A.rho + j);
        P.hm = __ldg(A.m + j);
        P.hw = ldw<WT>((c.halo < 0 ? A.w[0] : A.w[1]) + j);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (MSD >> a & 1) P.hmu[a] = __ldg(A.mu[a] + j);
    }
}

// late part: out-weights +x, -x, +y, -y, +z
template <typename WT, int MSD>
__device__ __forceinline__ void load_late(Pl<MSD>& P, const Ptrs<WT>& A, int zo, const Col& c) {
    if (!c.load) return;
    const int i = zo + c.o;
#pragma unroll
    for (int k = 0; k < 5; ++k) P.w[k] = ldw<WT>(A.w[k] + i);
}

template <int MSD>
__device__ __forceinline__ void zero_pl(Pl<MSD>& P) {
    P.r = 0.f;
    P.m = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) P.w[k] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) { P.mu[a] = 0.f; P.hmu[a] = 0.f; }
    P.hr = P.hw = 0.f;
    P.hm = make_float2(0.f, 0.f);
}

// Plane z: prefetch (early part of z+2 into pnn, late part and R of z+1),
// exchange x neighbours, update, store, accumulate.
template <typename WT, int MSD>
__device__ __forceinline__ void do_plane(const LatticeView& v, const Ptrs<WT>& A, const Col& c, int z, int z1,
                                         int plane, const Pl<MSD>& pb, const Pl<MSD>& pc, Pl<MSD>& pn,
                                         Pl<MSD>& pnn, const float2& Rc, float2& Rn, float* part) {
    if (z + 1 < z1) {
        int z2 = z + 2;
        while (z2 >= v.nz) z2 -= v.nz;
        const int zn = z + 1 >= v.nz ? z + 1 - v.nz : z + 1;
        load_early<WT, MSD>(pnn, A, z2 * plane, c);
        load_late<WT, MSD>(pn, A, zn * plane, c);
        if (c.load) Rn = __ldg(A.R + zn * plane + c.o);
    }
    const unsigned FULL = 0xffffffffu;
    SiteIn q;
    // the +x hop into this site comes from x-1 (lane-1), the -x hop from x+1
    q.r[0] = __shfl_up_sync(FULL, pc.r, 1);
    q.m[0].x = __shfl_up_sync(FULL, pc.m.x, 1);
    q.m[0].y = __shfl_up_sync(FULL, pc.m.y, 1);
    q.win[0] = __shfl_up_sync(FULL, pc.w[0], 1);
    q.r[1] = __shfl_down_sync(FULL, pc.r, 1);
    q.m[1].x = __shfl_down_sync(FULL, pc.m.x, 1);
    q.m[1].y = __shfl_down_sync(FULL, pc.m.y, 1);
    q.win[1] = __shfl_down_sync(FULL, pc.w[1], 1);
    float xm_mu[3], xp_mu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (MSD >> a & 1) {
            xm_mu[a] = __shfl_up_sync(FULL, pc.mu[a], 1);
            xp_mu[a] = __shfl_down_sync(FULL, pc.mu[a], 1);
        }
    if (c.lane == 0) {
        q.r[0] = pc.hr; q.m[0] = pc.hm; q.win[0] = pc.hw;
#pragma unroll
        for (int a = 0; a < 3; ++a) if (MSD >> a & 1) xm_mu[a] = pc.hmu[a];
    }
    if (c.lane == BX - 1) {
        q.r[1] = pc.hr; q.m[1] = pc.hm; q.win[1] = pc.hw;
#pragma unroll
        for (int a = 0; a < 3; ++a) if (MSD >> a & 1) xp_mu[a] = pc.hmu[a];
    }
    if (!c.site) return;
    const int zo = z * plane;
    const int i = zo + c.o;
    // y neighbours: +y hop from y-1, -y hop from y+1 (L1 / L2)
    q.r[2] = __ldg(A.rho + i - v.Xp);
    q.m[2] = __ldg(A.m + i - v.Xp);
    q.win[2] = ldw<WT>(A.w[2] + i - v.Xp);
    q.r[3] = __ldg(A.rho + i + v.Xp);
    q.m[3] = __ldg(A.m + i + v.Xp);
    q.win[3] = ldw<WT>(A.w[3] + i + v.Xp);
    // z neighbours from the register pipeline
    q.r[4] = pb.r; q.m[4] = pb.m; q.win[4] = pb.w[4];
    q.r[5] = pn.r; q.m[5] = pn.m; q.win[5] = pn.w[5];
#pragma unroll
    for (int k = 0; k < 6; ++k) q.wout[k] = pc.w[k];
    q.rc = pc.r;
    q.mc = pc.m;
    q.R = Rc;
    const float s = stay_weight(pc.w);
    float ro;
    float2 mo;
    site_rho_m(q, s, ro, mo);
    const long long zoff = (long long)zo;
    store_images(v.rho_out, v, c.x, c.y, zoff, ro);
    store_images(v.m_out, v, c.x, c.y, zoff, mo);
    part[0] += mo.x;
    part[1] += mo.y;
    part[2] += ro;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(MSD >> a & 1)) continue;
        const float nb[6] = {xm_mu[a], xp_mu[a], __ldg(A.mu[a] + i - v.Xp), __ldg(A.mu[a] + i + v.Xp),
                             pb.mu[a], pn.mu[a]};
        const float mo_a = site_mu(q.win, q.r, nb, s, pc.mu[a], a);
        store_images(v.mu_out[a], v, c.x, c.y, zoff, mo_a);
        part[3 + a] += site_dmsd(pc.w, pc.mu[a], pc.r, a);
    }
}

// One work item: the 32 x 8 tile (x-tile, y-tile) over planes
// [zc*cz, zc*cz+cz).  Adds this thread's site sums to part[] (FP32).
template <typename WT, int MSD>
__device__ __forceinline__ void step1_item(const LatticeView& v, int cz, int tiles_x, int tiles_y,
                                           int item, float* part) {
    const Ptrs<WT> A = make_ptrs<WT>(v);
    const int plane = v.Xp * v.Yp;
    const int tx = item % tiles_x;
    const int rest = item / tiles_x;
    const int tyi = rest % tiles_y;
    const int zc = rest / tiles_y;
    Col c;
    c.lane = threadIdx.x;
    c.x = tx * TX + threadIdx.x;
    c.y = tyi * TY + threadIdx.y;
    // a thread loads if its site is a lattice site or the ghost column right
    // of the lattice (the -x hop source of the previous lane's site)
    c.load = c.x <= v.nx && c.y < v.ny;
    c.site = c.x < v.nx && c.y < v.ny;
    c.halo = 0;
    if (c.load && c.lane == 0) c.halo = -1;
    if (c.site && c.lane == BX - 1) c.halo = 1;
    c.o = (c.y + v.G) * v.Xp + (c.x + v.G);
    const int z0 = v.zlo + zc * cz;
    const int z1 = min(z0 + cz, v.zhi);

    Pl<MSD> P0, P1, P2, P3;
    zero_pl(P0); zero_pl(P1); zero_pl(P2); zero_pl(P3);
    float2 R0 = make_float2(1.f, 0.f), R1 = R0;
    {
        const int zb = z0 == 0 ? v.nz - 1 : z0 - 1;
        const int zn = z0 + 1 >= v.nz ? z0 + 1 - v.nz : z0 + 1;
        load_early<WT, MSD>(P0, A, zb * plane, c);          // below: state, w4
        if (c.load) P0.w[4] = ldw<WT>(A.w[4] + zb * plane + c.o);
        load_early<WT, MSD>(P1, A, z0 * plane, c);          // this plane: everything
        load_late<WT, MSD>(P1, A, z0 * plane, c);
        load_early<WT, MSD>(P2, A, zn * plane, c);          // above: early part
        if (c.load) R0 = __ldg(A.R + z0 * plane + c.o);
    }
    // register sets rotate (below, at, above, prefetch): 0 1 2 3 -> 1 2 3 0 ...
    for (int z = z0; z < z1; z += 4) {
        do_plane<WT, MSD>(v, A, c, z, z1, plane, P0, P1, P2, P3, R0, R1, part);
        if (z + 1 >= z1) break;
        do_plane<WT, MSD>(v, A, c, z + 1, z1, plane, P1, P2, P3, P0, R1, R0, part);
        if (z + 2 >= z1) break;
        do_plane<WT, MSD>(v, A, c, z + 2, z1, plane, P2, P3, P0, P1, R0, R1, part);
        if (z + 3 >= z1) break;
        do_plane<WT, MSD>(v, A, c, z + 3, z1, plane, P3, P0, P1, P2, R1, R0, part);
    }
}

template <typename WT, int MSD>
__global__ void __launch_bounds__(BX * BY, 2)
k_step1(LatticeView v, int cz, int tiles_x, int tiles_y, int n_items) {
    __shared__ double smem[NWARP * kNumSums];
    const int lane = threadIdx.x;
    double acc[1][kNumSums] = {{0, 0, 0, 0, 0, 0}};
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        float part[kNumSums] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        step1_item<WT, MSD>(v, cz, tiles_x, tiles_y, item, part);
        // one FP32 warp reduction per item, accumulated in FP64 by lane 0
#pragma unroll
        for (int qq = 0; qq < kNumSums; ++qq) {
            if (qq >= 3 && !(MSD >> (qq - 3) & 1)) continue;
            const float t = warp_sum_f32(part[qq]);
            if (lane == 0) acc[0][qq] += (double)t;
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
    s.tiles_x = (v.nx + TX - 1) / TX;
    s.tiles_y = (v.ny + TY - 1) / TY;
    static int occ_cache[2][8] = {{0}};
    int& occ = occ_cache[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][v.msd_axes & 7];
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step1_kernel(wdtype, v.msd_axes), BX * BY, 0);
        if (occ < 1) occ = 1;
    }
    const long long resident = (long long)device_props().sm_count * occ;
    // z chunks: enough work items for ~8 waves, chunks of czmin..64 planes.
    // Small lattices are latency-bound (their state sits in L2): short chunks
    // put more blocks to work at the cost of re-reading two halo planes per
    // chunk (measured per step: 24^3 12.8 -> 6.8 us with 2 planes, 64^3
    // 13.6 -> 10.3 us and 96^3 24.6 -> 20.8 us with 4, against 8).
    const long long xy = (long long)s.tiles_x * s.tiles_y;
    const long long want = resident * 8;
    const long long nchunks = (want + xy - 1) / xy;
    const int nzu = v.zhi - v.zlo;              // planes updated
    const long long nsites = (long long)v.nx * v.ny * nzu;
    const int czmin = nsites < (1LL << 17) ? 2 : (nsites < (1LL << 21) ? 4 : 8);
    int cz = (int)((nzu + nchunks - 1) / nchunks);
    if (cz > 64) cz = 64;
    if (cz < czmin) cz = czmin;
    if (cz > nzu) cz = nzu;
    s.cz = cz;
    const long long nzc = (nzu + cz - 1) / cz;
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

// ---------------------------------------------------------------------------
// Batched launches: many lattices advance one step in one launch.
//
// Work items are the same 32 x 8 x cz tiles as above, with a fixed cz per
// lattice (kBatchCZ), listed lattice after lattice.  Each item's sums are
// combined in the block in a fixed order and stored in the lattice's own
// partials buffer at the item's index; the block that completes a lattice's
// last item sums that lattice's item partials in item order.  A lattice's
// results therefore do not depend on which other lattices share the launch.

namespace {

// One work item of a batched step: the tile's update, its sums combined in
// the block in a fixed order and stored at the item's index, and, in the
// block that completes the lattice's last item, the lattice's sums in item
// order.  V is the lattice's view for this step (input and output buffers).
template <typename WT, int MSD>
__device__ __forceinline__ void batch_item(const LatticeView& V, const BatchEntry& E, int li) {
    __shared__ double wsum[NWARP][kNumSums];
    __shared__ unsigned int last;
    const int lane = threadIdx.x;
    const int warp = threadIdx.y;
    const int tid = threadIdx.y * BX + threadIdx.x;
    float part[kNumSums] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    step1_item<WT, MSD>(V, E.cz, E.tiles_x, E.tiles_y, li, part);
#pragma unroll
    for (int qq = 0; qq < kNumSums; ++qq) {
        const float t = warp_sum_f32(part[qq]);
        if (lane == 0) wsum[warp][qq] = (double)t;
    }
    __syncthreads();
    if (tid < kNumSums) {
        double sacc = 0.0;
        for (int w = 0; w < NWARP; ++w) sacc += wsum[w][tid];
        V.partials[(long long)li * kNumSums + tid] = sacc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(V.counter, 1u) == (unsigned)E.n_items - 1u;
    __syncthreads();
    if (last) {
        __threadfence();
        const long long n = *V.step;
        if (warp < kNumSums) {
            const int q = warp;
            double sacc = 0.0;
            for (int b = lane; b < E.n_items; b += 32) sacc += __ldcg(&V.partials[(long long)b * kNumSums + q]);
            sacc = warp_sum_f64(sacc);
            if (lane == 0) {
                if (q == 0) V.histM[n + 1].x = sacc;
                else if (q == 1) V.histM[n + 1].y = sacc;
                else if (q == 2) V.histP[n + 1] = sacc;
                else if (MSD >> (q - 3) & 1) V.histD[(long long)(q - 3) * V.cap + n] = sacc;
            }
        }
        __syncthreads();
        if (tid == 0) {
            *V.step = n + 1;
            *V.counter = 0u;
        }
    }
    __syncthreads();
}

// Entry of a global item among the first `count` entries (items listed
// lattice after lattice).
__device__ __forceinline__ int batch_entry_of(const BatchParams& bp, int count, int gi) {
    int lo_ = 0, hi_ = count - 1;
    while (lo_ < hi_) {
        const int mid = (lo_ + hi_ + 1) >> 1;
        if (bp.e[mid].item0 <= gi) lo_ = mid;
        else hi_ = mid - 1;
    }
    return lo_;
}

template <typename WT, int MSD>
__global__ void __launch_bounds__(BX * BY, 2)
k_step_batch(const __grid_constant__ BatchParams bp) {
    for (int gi = blockIdx.x; gi < bp.total_items; gi += gridDim.x) {
        const BatchEntry& E = bp.e[batch_entry_of(bp, bp.count, gi)];
        batch_item<WT, MSD>(E.v, E, gi - E.item0);
    }
}

// The next step reads what this one wrote.
__device__ __forceinline__ void swap_io(LatticeView& v) {
    float* r = v.rho_out;
    v.rho_out = const_cast<float*>(v.rho_in);
    v.rho_in = r;
    float2* m = v.m_out;
    v.m_out = const_cast<float2*>(v.m_in);
    v.m_in = m;
    for (int a = 0; a < 3; ++a) {
        float* u = v.mu_out[a];
        v.mu_out[a] = const_cast<float*>(v.mu_in[a]);
        v.mu_in[a] = u;
    }
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr long long kGridWaitCycles = 2000000000LL;    // ~1 s at 2 GHz

// Grid-wide barrier of a cooperative launch: arrive on a counter, wait
// (bounded, with a short sleep) until all blocks of this phase arrived.
// Returns false when the wait ran out.
__device__ bool grid_sync_bounded(unsigned int* bar, unsigned int target) {
    __shared__ int bad;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        bad = 0;
        __threadfence();
        atomicAdd(bar, 1u);
        const long long t0 = clock64();
        while (ld_acquire(bar) < target) {
            if (clock64() - t0 > kGridWaitCycles) { bad = 1; break; }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return bad == 0;
}

// Persistent batched launch: every lattice advances its own number of steps
// (entries sorted by step count, descending, so the lattices still running at
// step t are a prefix), with a grid-wide barrier between steps.  Must be a
// cooperative launch.  A barrier that runs out records LPC_ERR_TIMEOUT in
// every lattice's error word and ends the launch.
template <typename WT, int MSD>
__global__ void __launch_bounds__(BX * BY, 2)
k_step_batch_multi(const __grid_constant__ BatchParams bp, int nsteps, unsigned int* bar) {
    for (int t = 0; t < nsteps; ++t) {
        int A = bp.count;
        while (A > 0 && bp.e[A - 1].steps <= t) --A;
        const int total = A == bp.count ? bp.total_items : bp.e[A].item0;
        for (int gi = blockIdx.x; gi < total; gi += gridDim.x) {
            const BatchEntry& E = bp.e[batch_entry_of(bp, A, gi)];
            LatticeView V = E.v;
            if (t & 1) swap_io(V);
            batch_item<WT, MSD>(V, E, gi - E.item0);
        }
        if (t + 1 < nsteps && !grid_sync_bounded(bar, (unsigned)(t + 1) * gridDim.x)) {
            if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
                for (int i = 0; i < bp.count; ++i) atomicExch(bp.e[i].v.counter + 1, (unsigned int)LPC_ERR_TIMEOUT);
            return;
        }
    }
}

template <typename WT, int MSD>
void* batch_fn() { return reinterpret_cast<void*>(&k_step_batch<WT, MSD>); }

void* batch_kernel(int wdtype, int msd) {
    static void* tab[2][8] = {
        {batch_fn<float, 0>(), batch_fn<float, 1>(), batch_fn<float, 2>(), batch_fn<float, 3>(),
         batch_fn<float, 4>(), batch_fn<float, 5>(), batch_fn<float, 6>(), batch_fn<float, 7>()},
        {batch_fn<__nv_bfloat16, 0>(), batch_fn<__nv_bfloat16, 1>(), batch_fn<__nv_bfloat16, 2>(),
         batch_fn<__nv_bfloat16, 3>(), batch_fn<__nv_bfloat16, 4>(), batch_fn<__nv_bfloat16, 5>(),
         batch_fn<__nv_bfloat16, 6>(), batch_fn<__nv_bfloat16, 7>()}};
    return tab[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
}


template <typename WT, int MSD>
void* batch_multi_fn() { return reinterpret_cast<void*>(&k_step_batch_multi<WT, MSD>); }

void* batch_multi_kernel(int wdtype, int msd) {
    static void* tab[2][8] = {
        {batch_multi_fn<float, 0>(), batch_multi_fn<float, 1>(), batch_multi_fn<float, 2>(),
         batch_multi_fn<float, 3>(), batch_multi_fn<float, 4>(), batch_multi_fn<float, 5>(),
         batch_multi_fn<float, 6>(), batch_multi_fn<float, 7>()},
        {batch_multi_fn<__nv_bfloat16, 0>(), batch_multi_fn<__nv_bfloat16, 1>(), batch_multi_fn<__nv_bfloat16, 2>(),
         batch_multi_fn<__nv_bfloat16, 3>(), batch_multi_fn<__nv_bfloat16, 4>(), batch_multi_fn<__nv_bfloat16, 5>(),
         batch_multi_fn<__nv_bfloat16, 6>(), batch_multi_fn<__nv_bfloat16, 7>()}};
    return tab[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
}

}  // namespace


int batch_items(const LatticeView& v, int* tiles_x, int* tiles_y, int* cz) {
    *tiles_x = (v.nx + TX - 1) / TX;
    *tiles_y = (v.ny + TY - 1) / TY;
    // chunk length from the lattice alone (so its sums do not depend on the
    // other lattices of a launch): short chunks for small, latency-bound lattices
    const long long nsites = (long long)v.nx * v.ny * v.nz;
    const int c = nsites < (1LL << 17) ? 2 : (nsites < (1LL << 20) ? 4 : kBatchCZ);
    *cz = v.nz < c ? v.nz : c;
    return *tiles_x * *tiles_y * ((v.nz + *cz - 1) / *cz);
}

cudaError_t launch_batch(const BatchParams& bp, int wdtype, int msd, cudaStream_t st) {
    void* fn = batch_kernel(wdtype, msd);
    static int occ_cache[2][8] = {{0}};
    int& occ = occ_cache[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BX * BY, 0);
        if (occ < 1) occ = 1;
    }
    int grid = device_props().sm_count * occ;
    if (grid > bp.total_items) grid = bp.total_items;
    if (grid < 1) return cudaSuccess;
    void* args[] = {const_cast<BatchParams*>(&bp)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(BX, BY), args, 0, st);
}

}  // namespace lpc

namespace lpc {

cudaError_t launch_batch_multi(const BatchParams& bp, int wdtype, int msd, int nsteps, unsigned int* bar,
                               cudaStream_t st) {
    void* fn = batch_multi_kernel(wdtype, msd);
    static int occ_cache[2][8] = {{0}};
    int& occ = occ_cache[wdtype == LPC_WEIGHTS_BF16 ? 1 : 0][msd & 7];
    if (occ == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, BX * BY, 0);
        if (occ < 1) occ = 1;
    }
    // every block must be resident (grid barrier): at most occupancy x SMs
    int grid = device_props().sm_count * occ;
    if (grid > bp.total_items) grid = bp.total_items;
    if (grid < 1 || nsteps < 1) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int ns = nsteps;
    unsigned int* b = bar;
    void* args[] = {const_cast<BatchParams*>(&bp), &ns, &b};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BX, BY), args, 0, st);
}

}  // namespace lpc
