// C ABI of the lattice-propagation library: handle lifetime, validation,
// device memory through the caller's allocator, the step schedule (direct
// launches or replay of captured CUDA graphs), history buffers and queries.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lpc_internal.cuh"

#define LPC_VERSION "lpc3d-b300 0.1 (sm_103a)"

namespace lpc {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

lpc_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return LPC_ERR_CUDA;
}

const DeviceProps& device_props() {
    static DeviceProps props[64];
    static bool init[64] = {false};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!init[dev]) {
        cudaDeviceGetAttribute(&props[dev].sm_count, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&props[dev].max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (props[dev].sm_count < 1) props[dev].sm_count = 1;
        init[dev] = true;
    }
    return props[dev];
}

}  // namespace lpc

namespace lpc {
// Both state buffers from the current rho: rho copied, m = rho, mu = 0
// (v: input = the current buffer); in kernels_pack.cu.
cudaError_t launch_restart(const LatticeView& v, cudaStream_t st);
// The value checks of create on the uploaded copies (F and rho0 finite on
// pore sites, omega finite, link factors in [0, 1]), or-ed as bits 0..3 into
// *bits (zeroed before); in kernels_pack.cu.
cudaError_t launch_check_inputs(const double* F, const double* omega, const uint8_t* solid, const double* rho0,
                                const double* links, long long N, unsigned int* bits, cudaStream_t st);
// Counter-block word of the input checks.
constexpr int kInputCheckWord = 30;
}  // namespace lpc

using namespace lpc;

struct lpc_lattice {
    lpc_params p;
    int G = 1, Xp = 0, Yp = 0;
    long long N = 0, Np = 0;
    int device = 0;
    cudaStream_t ustream = nullptr;     // the caller's stream
    cudaStream_t wstream = nullptr;     // private stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    lpc_allocator alloc{};
    bool user_alloc = false;
    long long device_bytes = 0;

    float* rho[2] = {nullptr, nullptr};
    float2* m[2] = {nullptr, nullptr};
    float* mu[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    void* w = nullptr;
    float2* R = nullptr;
    uint8_t* solid = nullptr;
    double2* histM = nullptr;
    double* histP = nullptr;
    double* histD = nullptr;
    long long cap = 0;
    double* partials = nullptr;
    size_t partials_doubles = 0;
    unsigned int* counter = nullptr;    // [0] completion counter, [2..3] step counter (int64)
    long long* dstep = nullptr;
    double* scratch = nullptr;          // small device scratch (Boltzmann sums, maxdiff)

    int cur = 0;
    long long steps = 0;
    int kernel = LPC_KERNEL_STEP1;
    int kdepth = 1;
    TBMaps* maps[2] = {nullptr, nullptr};   // TMA tensor maps per input parity
    int maps_K = 0;
    // gather form of the static data (one-step TMA kernel), made on first use
    void* gwin = nullptr;
    float* gs = nullptr;
    float2* gR = nullptr;
    void* gdm = nullptr;
    void* gdx = nullptr;                // inside the gwin block
    int Xs = 0;
    long long Ns = 0;
    // link form of the static data (plain lattices), instead of the gather form
    void* lnk = nullptr;
    void* lnk_x0 = nullptr;             // inside the lnk block
    size_t lnk_bytes = 0;
    int ny1 = 0;
    float link_a = 0.0f;
    bool links_given = false;           // created with per-link jump factors
    int static_pref = LPC_STATIC_AUTO;  // lattice_set_static_form
    // slab of a z-decomposed lattice (lattice_create_slab): planes 0 and
    // nz - 1 are halos, [zlo, zhi) the slab's own planes; a whole lattice has
    // zlo = 0, zhi = nz
    bool slab = false;
    int zlo = 0, zhi = 0;
    // tiling of the TMA-fed one-step kernel (lattice_set_tiling, autotuner): 0 = heuristic
    int t1_ty = 0, t1_ipc = 0;

    // captured step sequences: [parity] -> graph of graph_len steps
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_len = 0;

    // reservoir faces and region labels (lattice_create_ex)
    ResFaces rf{};
    uint8_t* region = nullptr;          // [nz][ny][Xr]
    int nreg = 0;
    int Xr = 0;
    double* rpart = nullptr;            // per-block partials of the region pass
};

namespace {

// NVTX range over one ABI call (host timeline of nsys / ncu --nvtx; a no-op
// when no tool is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct Entry {
    // Orders the private stream after the caller's stream on entry and the
    // caller's stream after the private stream on exit.
    lpc_lattice* h;
    explicit Entry(lpc_lattice* hh) : h(hh) {
        cudaSetDevice(h->device);
        cudaEventRecord(h->ev_in, h->ustream);
        cudaStreamWaitEvent(h->wstream, h->ev_in, 0);
    }
    ~Entry() {
        cudaEventRecord(h->ev_out, h->wstream);
        cudaStreamWaitEvent(h->ustream, h->ev_out, 0);
    }
};

void* dalloc(lpc_lattice* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (h->user_alloc) {
        p = h->alloc.alloc(bytes, (void*)h->ustream, h->alloc.ctx);
    } else {
        if (cudaMallocAsync(&p, bytes, h->wstream) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) h->device_bytes += (long long)bytes;
    return p;
}

void dfree(lpc_lattice* h, void* p, size_t bytes) {
    if (!p) return;
    if (h->user_alloc) h->alloc.free(p, (void*)h->ustream, h->alloc.ctx);
    else cudaFreeAsync(p, h->wstream);
    h->device_bytes -= (long long)bytes;
}

size_t wbytes(const lpc_lattice* h) { return h->p.weight_dtype == LPC_WEIGHTS_BF16 ? 2 : 4; }

// One history set is M (double2), P and dMSD x, y, z per step; a lattice
// holds the totals and one set per region, laid out [set][cap] per quantity.
size_t history_bytes(long long cap, int sets) {
    return (size_t)cap * sets * (sizeof(double2) + sizeof(double) * 4);
}

// Steps of a TB launch that this lattice may use: reservoir ghosts must keep
// their values and region sums are taken once per step, so lattices with
// either run one step per launch.
bool tb_depth_allowed(const lpc_lattice* h, int K) { return K == 1 || (!h->rf.any() && h->nreg == 0 && !h->slab); }

LatticeView make_view(lpc_lattice* h, int in) {
    LatticeView v;
    v.nx = h->p.nx; v.ny = h->p.ny; v.nz = h->p.nz;
    v.zlo = h->zlo; v.zhi = h->zhi;
    v.G = h->G; v.Xp = h->Xp; v.Yp = h->Yp;
    v.per_x = h->p.periodic[0]; v.per_y = h->p.periodic[1]; v.per_z = h->p.periodic[2];
    v.msd_axes = h->p.msd_axes;
    v.Np = h->Np;
    v.rho_in = h->rho[in]; v.m_in = h->m[in];
    v.rho_out = h->rho[in ^ 1]; v.m_out = h->m[in ^ 1];
    for (int a = 0; a < 3; ++a) { v.mu_in[a] = h->mu[in][a]; v.mu_out[a] = h->mu[in ^ 1][a]; }
    v.w = h->w; v.R = h->R;
    v.gwin = h->gwin; v.gs = h->gs; v.gR = h->gR; v.gdm = h->gdm; v.gdx = h->gdx; v.Xs = h->Xs; v.Ns = h->Ns;
    v.lnk = h->lnk; v.lnk_x0 = h->lnk_x0; v.ny1 = h->ny1; v.link_a = h->link_a;
    v.partials = h->partials; v.counter = h->counter; v.step = h->dstep;
    v.histM = h->histM; v.histP = h->histP; v.histD = h->histD; v.cap = h->cap;
    v.region = h->region; v.nreg = h->nreg; v.Xr = h->Xr;
    v.t1_ty = h->t1_ty; v.t1_ipc = h->t1_ipc;
    return v;
}

// Sites a step updates (a slab's own planes, without its halos).
long long n_updated(const lpc_lattice* h) { return (long long)h->p.nx * h->p.ny * (h->zhi - h->zlo); }

// The view of the planes [zlo, zhi) alone, as a lattice of zhi - zlo planes
// (per-plane pointers offset, plane strides unchanged): for the reductions
// and read-backs that walk every plane of a view.
LatticeView updated_view(lpc_lattice* h, int in) {
    LatticeView v = make_view(h, in);
    const long long off = (long long)h->zlo * h->Xp * h->Yp;
    if (off == 0) return v;
    v.nz = h->zhi - h->zlo;
    v.zlo = 0;
    v.zhi = v.nz;
    v.rho_in += off; v.m_in += off; v.rho_out += off; v.m_out += off;
    for (int a = 0; a < 3; ++a) {
        if (v.mu_in[a]) v.mu_in[a] += off;
        if (v.mu_out[a]) v.mu_out[a] += off;
    }
    v.w = static_cast<const char*>(v.w) + off * (long long)wbytes(h);
    v.R += off;
    if (v.region) v.region += (long long)h->zlo * h->p.ny * h->Xr;
    return v;
}

void drop_graphs(lpc_lattice* h) {
    for (int i = 0; i < 2; ++i)
        if (h->graph[i]) { cudaGraphExecDestroy(h->graph[i]); h->graph[i] = nullptr; }
    h->graph_len = 0;
}

lpc_status ensure_history(lpc_lattice* h, long long needed) {
    if (needed <= h->cap) return LPC_OK;
    long long ncap = h->cap * 2;
    if (ncap < needed) ncap = needed;
    if (ncap < 1024) ncap = 1024;
    const int sets = 1 + h->nreg;
    char* blk = (char*)dalloc(h, history_bytes(ncap, sets));
    if (!blk) { set_error("history allocation failed"); return LPC_ERR_OOM; }
    double2* nM = (double2*)blk;
    double* nP = (double*)(blk + sizeof(double2) * ncap * sets);
    double* nD = nP + ncap * sets;
    cudaError_t e = cudaMemsetAsync(blk, 0, history_bytes(ncap, sets), h->wstream);
    for (int st = 0; st < sets && e == cudaSuccess && h->cap > 0; ++st) {
        e = cudaMemcpyAsync(nM + st * ncap, h->histM + st * h->cap, sizeof(double2) * h->cap,
                            cudaMemcpyDeviceToDevice, h->wstream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(nP + st * ncap, h->histP + st * h->cap, sizeof(double) * h->cap,
                                cudaMemcpyDeviceToDevice, h->wstream);
        for (int a = 0; a < 3 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(nD + (st * 3 + a) * ncap, h->histD + (st * 3 + a) * h->cap,
                                sizeof(double) * h->cap, cudaMemcpyDeviceToDevice, h->wstream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "history copy");
    if (h->histM) {
        // the old block must not be reused before the copies above finish
        cudaStreamSynchronize(h->wstream);
        dfree(h, h->histM, history_bytes(h->cap, sets));
    }
    h->histM = nM; h->histP = nP; h->histD = nD; h->cap = ncap;
    drop_graphs(h);
    return LPC_OK;
}

// Bytes of the x out-weights at the tile edges ([nz][tiles_x][nyp][2]).
size_t gather_dx_bytes(const lpc_params& p) {
    const size_t wb = p.weight_dtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    return ((size_t)p.nz * ((p.nx + 63) / 64) * ((p.ny + 7) / 8 * 8) * 2 * wb + 255) / 256 * 256;
}

// win (6 planes), s, R and, with any MSD axis, one (w+a, w-a) plane per axis
// (the x pairs replaced by the tile-edge array)
size_t gather_bytes(long long Ns, const lpc_params& p, int msd) {
    const size_t wb = p.weight_dtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    return (size_t)Ns * (6 * wb + 4 + 8 + (msd ? 3 * 2 * wb : 0)) + ((msd & 1) ? gather_dx_bytes(p) : 0);
}

// The gather form keeps the MSD out-weight pairs only where the MSD sums are
// taken over source sites: with regions (the site's region at the step) or
// reservoir faces (hops into a reservoir count, hops out of one do not).
bool gather_dm(const lpc_lattice* h) { return h->p.msd_axes && (h->nreg > 0 || h->rf.any()); }

// The static data of the one-step TMA kernel, made once (outside any stream
// capture) from the padded weight planes: the link form for large plain
// lattices (one jump factor, no reservoir face, no regions: 12 + 8 bytes per
// site with FP32 weights, 6 + 8 with BF16), else the gather form (or when a
// link does not fit the link form).  The link form saves bytes but spends
// instructions rebuilding the weights; measured per site update with FP32
// weights it wins from about 50M sites (1.07e11 vs 1.09e11 site-updates/s at
// 384^3, 1.09e11 vs 1.27e11 at 512^3) and loses below (9.7e10 vs 9.2e10 at
// 256^3).  BF16 weights already make the gather form small (24 bytes per
// site); there the rebuild costs more than the bytes it saves (1.34e11 vs
// 1.25e11 on the 512^3 monolith), so BF16 lattices keep the gather form.
// Since the kernel pairs the FP32 arithmetic of a lane's two sites, the two
// forms are within a few per cent of each other where the rule switches:
// 9.72e10 (gather) vs 9.83e10 (link) at 256^3, and with BF16 weights
// 1.340e11 vs 1.326e11 on the 512^3 monolith, 1.126e11 vs 1.160e11 on the
// 2048x256x256 slab with the x moment; the rule is kept as it is.
constexpr long long kLinkFormSites = 3LL << 24;

// The link form holds the lattices with one jump factor (reservoir links take
// it too); per-link factors break its rule that one hop of every open link
// weighs alpha/6.
bool link_form_possible(const lpc_lattice* h) { return !h->links_given; }

lpc_status ensure_gather(lpc_lattice* h) {
    if (h->gwin || h->lnk) return LPC_OK;
    const int Xs = gather_pitch(h->p.nx);
    const long long Ns = (long long)Xs * h->p.ny * h->p.nz;
    const bool want_link =
        link_form_possible(h) &&
        (h->static_pref == LPC_STATIC_LINK ||
         (h->static_pref == LPC_STATIC_AUTO && n_updated(h) >= kLinkFormSites && h->p.weight_dtype == LPC_WEIGHTS_F32));
    if (want_link) {
        const int ny1 = h->p.ny + 1;
        const size_t lb = ((size_t)3 * h->p.nz * ny1 * Xs * wbytes(h) + 255) / 256 * 256;
        const size_t x0b = ((size_t)h->p.nz * h->p.ny * wbytes(h) + 255) / 256 * 256;
        const size_t bytes = lb + x0b + (size_t)Ns * 8;
        char* blk = (char*)dalloc(h, bytes);
        if (!blk && h->static_pref == LPC_STATIC_LINK) { set_error("link-form allocation failed"); return LPC_ERR_OOM; }
        if (blk) {
            h->Xs = Xs;
            h->ny1 = ny1;
            LatticeView v = make_view(h, h->cur);
            v.Xs = Xs;
            v.ny1 = ny1;
            void* X0 = blk + lb;
            float2* Rl = reinterpret_cast<float2*>(blk + lb + x0b);
            unsigned int* bad = reinterpret_cast<unsigned int*>(h->scratch);
            float* a_out = reinterpret_cast<float*>(h->scratch) + 1;
            cudaError_t e = cudaMemsetAsync(bad, 0, 4, h->wstream);
            if (e == cudaSuccess)
                e = launch_link_pack(v, h->p.weight_dtype, blk, X0, Rl, h->p.alpha, bad, a_out, h->wstream);
            unsigned int hb[2] = {1u, 0u};
            if (e == cudaSuccess) e = cudaMemcpyAsync(hb, bad, 8, cudaMemcpyDeviceToHost, h->wstream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
            if (e != cudaSuccess) { dfree(h, blk, bytes); return cuda_fail(e, "link pack"); }
            if (hb[0] == 0u) {
                h->lnk = blk;
                h->lnk_x0 = X0;
                h->lnk_bytes = bytes;
                h->gR = Rl;
                h->Ns = Ns;
                memcpy(&h->link_a, &hb[1], 4);
                return LPC_OK;
            }
            dfree(h, blk, bytes);     // a link outside the form: use the gather form
            h->ny1 = 0;
            if (h->static_pref == LPC_STATIC_LINK) {
                set_error("a link's weights do not fit the link form (one hop of every open link weighs alpha/6)");
                return LPC_ERR_STATE;
            }
        }
    }
    char* blk = (char*)dalloc(h, gather_bytes(Ns, h->p, gather_dm(h) ? h->p.msd_axes : 0));
    if (!blk) { set_error("gather-form allocation failed"); return LPC_ERR_OOM; }
    h->Xs = Xs;
    h->Ns = Ns;
    h->gwin = blk;
    blk += (size_t)Ns * 6 * wbytes(h);
    h->gs = (float*)blk;
    blk += (size_t)Ns * 4;
    h->gR = (float2*)blk;
    blk += (size_t)Ns * 8;
    h->gdm = gather_dm(h) ? (void*)blk : nullptr;       // [3][Ns][2] weights, indexed by axis
    blk += gather_dm(h) ? (size_t)Ns * 3 * 2 * wbytes(h) : 0;
    h->gdx = (gather_dm(h) && (h->p.msd_axes & 1)) ? (void*)blk : nullptr;
    LatticeView v = make_view(h, h->cur);
    cudaError_t e = launch_gather_pack(v, h->p.weight_dtype, h->gwin, h->gs, h->gR, h->gdm, h->gdx, h->wstream);
    if (e != cudaSuccess) return cuda_fail(e, "gather pack");
    return LPC_OK;
}

lpc_status ensure_maps(lpc_lattice* h) {
    if (h->kdepth == 1) {
        lpc_status g = ensure_gather(h);
        if (g != LPC_OK) return g;
    }
    if (h->maps[0] && h->maps_K == h->kdepth) return LPC_OK;
    for (int par = 0; par < 2; ++par) {
        if (!h->maps[par]) h->maps[par] = tb_maps_new();
        if (!h->maps[par]) { set_error("tensor map allocation failed"); return LPC_ERR_OOM; }
        LatticeView v = make_view(h, par);
        int W = 0, H = 0;
        const bool ok = h->kdepth == 1
                            ? t1_encode_maps(v, h->p.weight_dtype, h->maps[par])
                            : tb_box_dims(v, h->p.weight_dtype, h->kdepth, &W, &H) &&
                                  tb_encode_maps(v, h->p.weight_dtype, W, H, h->maps[par]);
        if (!ok) {
            set_error("TMA tensor map encoding failed");
            return LPC_ERR_CUDA;
        }
    }
    h->maps_K = h->kdepth;
    return LPC_OK;
}

// One launch: a TB block of kdepth steps (tb = true) or one step.
lpc_status launch_one(lpc_lattice* h, cudaStream_t st, bool tb = false) {
    cudaError_t e;
    if (tb) {
        lpc_status s = ensure_maps(h);
        if (s != LPC_OK) return s;
        const LatticeView v = make_view(h, h->cur);
        e = launch_tb(v, h->p.weight_dtype, h->kdepth, *h->maps[h->cur], h->counter + 1, st);
    } else {
        e = launch_step1(make_view(h, h->cur), h->p.weight_dtype, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    h->cur ^= 1;
    // region sums: taken by the one-step TMA kernel itself where it can,
    // else by the separate pass over the new state
    if (h->nreg > 0 && !(tb && h->kdepth == 1 && t1_fused_regions(make_view(h, h->cur), h->p.weight_dtype))) {
        e = launch_region_sums(updated_view(h, h->cur), h->p.weight_dtype, h->rpart, h->counter + 12, false, st);
        if (e != cudaSuccess) return cuda_fail(e, "region sums launch");
    }
    return LPC_OK;
}

// Device error word (set by kernels whose bounded waits ran out).
lpc_status check_device_error(lpc_lattice* h) {
    unsigned int err = 0;
    cudaError_t e = cudaMemcpy(&err, h->counter + 1, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "error word read");
    if (err != 0) {
        cudaMemset(h->counter, 0, 8);   // completion counter and error word
        set_error("a device wait exceeded its time limit (kernel returned early)");
        return (lpc_status)err;
    }
    return LPC_OK;
}

constexpr int kGraphLen = 32;   // steps per captured graph (even: keeps buffer parity)

lpc_status build_graph(lpc_lattice* h, int parity) {
    cudaGraph_t g = nullptr;
    const bool tb = h->kernel == LPC_KERNEL_TB;
    if (tb) {
        // maps and gather-form arrays are made before the capture
        lpc_status s0 = ensure_maps(h);
        if (s0 != LPC_OK) return s0;
    }
    cudaError_t e = cudaStreamBeginCapture(h->wstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
    const int save = h->cur;
    h->cur = parity;
    lpc_status st = LPC_OK;
    for (int i = 0; i < kGraphLen && st == LPC_OK; ++i) st = launch_one(h, h->wstream, tb);
    h->cur = save;
    e = cudaStreamEndCapture(h->wstream, &g);
    if (st != LPC_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    e = cudaGraphInstantiate(&h->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    h->graph_len = kGraphLen;
    return LPC_OK;
}

// Default schedule: the TMA-fed one-step kernel for lattices large enough to
// fill its tiles, else the register-pipelined one-step kernel.
void auto_schedule(lpc_lattice* h) {
    const bool big = h->p.nx >= 64 && h->p.ny >= 16 && n_updated(h) >= (1LL << 20);
    if (big && tb_supported(make_view(h, 0), h->p.weight_dtype, 1) &&
        tb_prepare(h->p.weight_dtype, 1, h->p.msd_axes) == cudaSuccess) {
        h->kernel = LPC_KERNEL_TB;
        h->kdepth = 1;
    } else {
        h->kernel = LPC_KERNEL_STEP1;
        h->kdepth = 1;
    }
    drop_graphs(h);
}

// pred(i) for every i < n, on up to 16 host threads for large inputs (the
// argument checks of create read every input value once).
template <typename Pred>
bool all_of_parallel(long long n, Pred pred) {
    unsigned T = std::thread::hardware_concurrency();
    T = T < 1 ? 1 : (T > 16 ? 16 : T);
    if (n < (1LL << 20)) T = 1;
    std::atomic<bool> ok{true};
    auto part = [&](unsigned t) {
        const long long lo = n * t / T, hi = n * (t + 1) / T;
        for (long long i = lo; i < hi; ++i)
            if (!pred(i)) { ok.store(false, std::memory_order_relaxed); return; }
    };
    if (T == 1) {
        part(0);
        return ok.load();
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (unsigned t = 0; t < T; ++t) th.emplace_back(part, t);
    for (auto& x : th) x.join();
    return ok.load();
}

bool finite_all(const double* a, const uint8_t* solid, long long n, bool pore_only) {
    return all_of_parallel(n, [=](long long i) { return (pore_only && solid[i]) || std::isfinite(a[i]); });
}

// Release the static data of the one-step TMA kernel (either form); the next
// launch of that kernel makes it again.  Tensor maps and graphs that name it
// are dropped.
void drop_static(lpc_lattice* h) {
    if (!h->gwin && !h->lnk) return;
    cudaStreamSynchronize(h->wstream);
    drop_graphs(h);
    if (h->gwin) dfree(h, h->gwin, gather_bytes(h->Ns, h->p, gather_dm(h) ? h->p.msd_axes : 0));
    if (h->lnk) dfree(h, h->lnk, h->lnk_bytes);
    h->gwin = nullptr; h->gs = nullptr; h->gR = nullptr; h->gdm = nullptr; h->gdx = nullptr;
    h->lnk = nullptr; h->lnk_x0 = nullptr; h->lnk_bytes = 0; h->ny1 = 0; h->link_a = 0.0f;
    h->Xs = 0; h->Ns = 0;
    h->maps_K = 0;          // re-encode the tensor maps on the next launch
}

void release_all(lpc_lattice* h) {
    if (h->wstream) cudaStreamSynchronize(h->wstream);
    drop_graphs(h);
    const size_t Np = (size_t)h->Np;
    for (int b = 0; b < 2; ++b) {
        dfree(h, h->rho[b], Np * 4);
        dfree(h, h->m[b], Np * 8);
        for (int a = 0; a < 3; ++a) dfree(h, h->mu[b][a], Np * 4);
    }
    dfree(h, h->w, Np * 6 * wbytes(h));
    dfree(h, h->R, Np * 8);
    if (h->gwin) dfree(h, h->gwin, gather_bytes(h->Ns, h->p, gather_dm(h) ? h->p.msd_axes : 0));
    if (h->lnk) dfree(h, h->lnk, h->lnk_bytes);
    dfree(h, h->solid, (size_t)h->N);
    if (h->region) dfree(h, h->region, (size_t)h->Xr * h->p.ny * h->p.nz);
    if (h->rpart) dfree(h, h->rpart, (size_t)region_blocks() * LPC_MAX_REGIONS * 6 * 8);
    if (h->histM) dfree(h, h->histM, history_bytes(h->cap, 1 + h->nreg));
    dfree(h, h->partials, h->partials_doubles * 8);
    dfree(h, h->counter, 256);
    dfree(h, h->scratch, 8 * 1024);
    if (h->ustream) cudaStreamSynchronize(h->ustream);
    for (int i = 0; i < 2; ++i) if (h->maps[i]) tb_maps_delete(h->maps[i]);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->wstream) cudaStreamDestroy(h->wstream);
}

}  // namespace

extern "C" {

const char* lpc_last_error(void) { return g_err.c_str(); }

const char* lpc_version(void) { return LPC_VERSION; }

lpc_status lattice_create(const lpc_params* p, const double* F, const double* omega,
                          const uint8_t* solid, const double* rho0, const lpc_allocator* a,
                          void* stream, lpc_lattice** out) {
    return lattice_create_ex(p, nullptr, F, omega, solid, rho0, a, stream, out);
}

lpc_status lattice_create_links(const lpc_params* p, const double* F, const double* omega,
                                const uint8_t* solid, const double* rho0, const double* alpha_links,
                                const lpc_allocator* a, void* stream, lpc_lattice** out) {
    lpc_options o;
    memset(&o, 0, sizeof o);
    o.alpha_links = alpha_links;
    return lattice_create_ex(p, &o, F, omega, solid, rho0, a, stream, out);
}

}  // extern "C"

namespace {

enum CreateMode { kWhole = 0, kSlab = 1, kZHalos = 2 };

lpc_status create_with_z_halos(const lpc_params* p, const lpc_options& o, const double* F, const double* omega,
                               const uint8_t* solid, const double* rho0, const lpc_allocator* a, void* stream,
                               lpc_lattice** out);

// lattice_create_ex (kWhole), lattice_create_slab (kSlab: p->nz counts the
// two halo planes too), and a whole lattice with a reservoir on a z face
// (kZHalos: the reservoir sites are a halo plane, p->nz counts both halos).
lpc_status create_impl(const lpc_params* p, const lpc_options* opt, const double* F, const double* omega,
                       const uint8_t* solid, const double* rho0, const lpc_allocator* a, void* stream,
                       lpc_lattice** out, int mode) {
    const bool slab = mode == kSlab;
    Range nvtx("lattice_create");
    if (out) *out = nullptr;
    lpc_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    const double* alpha_links = o.alpha_links;
    if (!p || !F || !omega || !solid || !out) { set_error("lattice_create: NULL argument"); return LPC_ERR_INVALID; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { set_error("lattice_create: edges must be >= 1"); return LPC_ERR_INVALID; }
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N > 2147483647LL) { set_error("lattice_create: more than 2^31-1 sites"); return LPC_ERR_INVALID; }
    if (!(p->alpha > 0.0 && p->alpha <= 1.0)) { set_error("lattice_create: alpha must be in (0, 1]"); return LPC_ERR_INVALID; }
    if (!(p->kT > 0.0) || !std::isfinite(p->kT) || !std::isfinite(p->dt)) { set_error("lattice_create: kT must be > 0 and dt finite"); return LPC_ERR_INVALID; }
    if (p->weight_dtype != LPC_WEIGHTS_F32 && p->weight_dtype != LPC_WEIGHTS_BF16) { set_error("lattice_create: weight_dtype must be 0 (FP32) or 1 (BF16)"); return LPC_ERR_INVALID; }
    if (p->msd_axes < 0 || p->msd_axes > 7) { set_error("lattice_create: msd_axes must be a mask of 1, 2, 4"); return LPC_ERR_INVALID; }
    if (p->init != LPC_INIT_UNIFORM && p->init != LPC_INIT_BOLTZMANN) { set_error("lattice_create: init must be 0 or 1"); return LPC_ERR_INVALID; }
    if (p->ghost < 0 || p->ghost > kMaxGhost || (p->ghost & 1)) { set_error("lattice_create: ghost must be 0 (automatic) or even in 2..8"); return LPC_ERR_INVALID; }
    {
        // the kernels address the padded arrays with 32-bit offsets; checked
        // before any input array is read
        const long long Gp = p->ghost == 0 ? 2 : p->ghost;
        const long long Np = ((p->nx + 2 * Gp) + 31) / 32 * 32 * (p->ny + 2 * Gp) * (long long)p->nz;
        if (Np > 2147483647LL) {
            set_error("lattice_create: more than 2^31-1 sites including the ghost layers");
            return LPC_ERR_INVALID;
        }
    }
    for (int i = 0; i < 3; ++i)
        if (p->periodic[i] != 0 && p->periodic[i] != 1) { set_error("lattice_create: periodic flags must be 0 or 1"); return LPC_ERR_INVALID; }
    if (a && (!a->alloc || !a->free)) { set_error("lattice_create: allocator needs alloc and free"); return LPC_ERR_INVALID; }
    // the checks that read every input value: finite F and rho0 on pore
    // sites, finite omega, link factors in [0, 1]
    auto check_values = [=]() -> const char* {
        if (!finite_all(F, solid, N, true)) return "lattice_create: non-finite F on a pore site";
        if (!finite_all(omega, solid, N, false)) return "lattice_create: non-finite omega";
        if (rho0 && !finite_all(rho0, solid, N, true)) return "lattice_create: non-finite rho0 on a pore site";
        if (alpha_links && !all_of_parallel(3 * N, [=](long long i) { return alpha_links[i] >= 0.0 && alpha_links[i] <= 1.0; }))
            return "lattice_create_links: link factors must be in [0, 1]";
        return nullptr;
    };
    if (o.reserved != 0) { set_error("lattice_create_ex: reserved option fields must be 0"); return LPC_ERR_INVALID; }
    ResFaces rf{};
    for (int f = 0; f < 6; ++f) {
        const lpc_reservoir& r = o.reservoir[f];
        if (!r.enabled) continue;
        if (r.enabled != 1 || r.reserved != 0) { set_error("lattice_create_ex: reservoir.enabled must be 0 or 1 and reserved 0"); return LPC_ERR_INVALID; }
        if (f >= 4 && slab) { set_error("lattice_create_slab: a slab's z faces are its halo planes, not reservoirs"); return LPC_ERR_INVALID; }
        if (p->periodic[f >> 1]) { set_error("lattice_create_ex: a reservoir needs a non-periodic axis"); return LPC_ERR_INVALID; }
        if (!std::isfinite(r.F) || !std::isfinite(r.rho) || !std::isfinite(r.m_re) || !std::isfinite(r.m_im)) {
            set_error("lattice_create_ex: non-finite reservoir values");
            return LPC_ERR_INVALID;
        }
        rf.on[f] = 1;
        rf.F[f] = r.F;
        rf.rho[f] = (float)r.rho;
        rf.m[f] = make_float2((float)r.m_re, (float)r.m_im);
    }
    if ((o.region == nullptr) != (o.n_regions == 0) || o.n_regions < 0 || o.n_regions > LPC_MAX_REGIONS) {
        set_error("lattice_create_ex: n_regions must be 1..4 with region labels and 0 without");
        return LPC_ERR_INVALID;
    }
    if (slab && o.region) {
        set_error("lattice_create_slab: slabs take no region labels");
        return LPC_ERR_INVALID;
    }
    if (slab && !rho0 && p->init == LPC_INIT_BOLTZMANN) {
        set_error("lattice_create_slab: a Boltzmann start is normalised over the whole lattice: pass rho0");
        return LPC_ERR_INVALID;
    }
    if (o.region) {
        const uint8_t* reg = o.region;
        const int nr = o.n_regions;
        if (!all_of_parallel(N, [=](long long i) { return reg[i] < nr; })) {
            set_error("lattice_create_ex: a region label is >= n_regions");
            return LPC_ERR_INVALID;
        }
    }
    // the extended fields of a z reservoir are checked by the call that takes them
    if (mode == kWhole && rf.any_z()) return create_with_z_halos(p, o, F, omega, solid, rho0, a, stream, out);
    // Small lattices are checked on the host before any device work.  A large
    // lattice's values are checked on the device, in its uploaded copies (a
    // host scan of gigabytes cost as much as the upload and the pack
    // together); a failure releases everything made so far and returns
    // LPC_ERR_INVALID, as the host check does.
    const bool device_check = N >= (1LL << 22);
    if (!device_check) {
        const char* bad = check_values();
        if (bad) { set_error(bad); return LPC_ERR_INVALID; }
    }

    lpc_lattice* h = new (std::nothrow) lpc_lattice();
    if (!h) { set_error("lattice_create: host allocation failed"); return LPC_ERR_OOM; }
    h->p = *p;
    h->N = N;
    h->slab = slab;
    h->zlo = mode == kWhole ? 0 : 1;
    h->zhi = mode == kWhole ? p->nz : p->nz - 1;
    h->rf = rf;
    h->links_given = alpha_links != nullptr;
    h->nreg = o.n_regions;
    h->Xr = gather_pitch(p->nx);
    cudaGetDevice(&h->device);
    int G = p->ghost;
    if (G == 0) G = 2;
    h->G = G;
    h->Xp = ((p->nx + 2 * G) + 31) / 32 * 32;     // rows start on 128-byte lines
    h->Yp = p->ny + 2 * G;
    h->Np = (long long)h->Xp * h->Yp * p->nz;
    if (h->Np > 2147483647LL) {
        // the kernels address the padded arrays with 32-bit offsets
        delete h;
        set_error("lattice_create: more than 2^31-1 sites including the ghost layers");
        return LPC_ERR_INVALID;
    }
    h->ustream = (cudaStream_t)stream;
    if (a) { h->alloc = *a; h->user_alloc = true; }

    cudaError_t e = cudaStreamCreateWithFlags(&h->wstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) { lpc_status s = cuda_fail(e, "lattice_create: stream setup"); release_all(h); delete h; return s; }

    const size_t Np = (size_t)h->Np;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && (h->rho[b] = (float*)dalloc(h, Np * 4));
        ok = ok && (h->m[b] = (float2*)dalloc(h, Np * 8));
        for (int ax = 0; ax < 3 && ok; ++ax)
            if (p->msd_axes >> ax & 1) ok = ok && (h->mu[b][ax] = (float*)dalloc(h, Np * 4));
    }
    ok = ok && (h->w = dalloc(h, Np * 6 * wbytes(h)));
    ok = ok && (h->R = (float2*)dalloc(h, Np * 8));
    ok = ok && (h->solid = (uint8_t*)dalloc(h, (size_t)N));
    // per-item sums of the one-step kernels: the totals, and with regions each region's
    h->partials_doubles = (size_t)device_props().sm_count * 32 * kMaxTB * kNumSums *
                          (o.region ? 1 + LPC_MAX_REGIONS : 1);
    ok = ok && (h->partials = (double*)dalloc(h, h->partials_doubles * 8));
    ok = ok && (h->counter = (unsigned int*)dalloc(h, 256));
    ok = ok && (h->scratch = (double*)dalloc(h, 8 * 1024));
    const size_t region_bytes = (size_t)h->Xr * p->ny * p->nz;
    if (o.region) {
        ok = ok && (h->region = (uint8_t*)dalloc(h, region_bytes));
        ok = ok && (h->rpart = (double*)dalloc(h, (size_t)region_blocks() * LPC_MAX_REGIONS * 6 * 8));
    }
    // temporaries for the inputs
    double* dF = nullptr; double* dO = nullptr; double* dR0 = nullptr; double* dA = nullptr;
    ok = ok && (dF = (double*)dalloc(h, (size_t)N * 8));
    ok = ok && (dO = (double*)dalloc(h, (size_t)N * 8));
    if (ok && rho0) ok = (dR0 = (double*)dalloc(h, (size_t)N * 8)) != nullptr;
    if (ok && alpha_links) ok = (dA = (double*)dalloc(h, (size_t)N * 24)) != nullptr;
    if (!ok) {
        set_error("lattice_create: device allocation failed");
        dfree(h, dF, (size_t)N * 8); dfree(h, dO, (size_t)N * 8); dfree(h, dR0, (size_t)N * 8);
        dfree(h, dA, (size_t)N * 24);
        release_all(h); delete h;
        return LPC_ERR_OOM;
    }
    h->dstep = reinterpret_cast<long long*>(h->counter + 2);
    lpc_status st = LPC_OK;
    {
        Entry en(h);
        const long long minus_one = -1;
        e = cudaMemsetAsync(h->counter, 0, 256, h->wstream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->dstep, &minus_one, 8, cudaMemcpyHostToDevice, h->wstream);
        // Large lattices without per-link factors upload F, omega and the
        // mask in chunks of planes and pack each chunk on a second stream as
        // soon as the chunk above it has arrived (a plane's weights read its
        // own and its z neighbours' fields), so the pack overlaps the upload;
        // the last chunk's arrival also releases the chunks that wrap in z.
        const LatticeView pv = make_view(h, 1);    // the pack writes the static planes
        const long long uplane = (long long)p->nx * p->ny;
        const int nchunk = (!alpha_links && N >= (1LL << 22)) ? std::min(8, p->nz) : 1;
        cudaStream_t ps = nullptr;
        cudaEvent_t pev[9] = {};
        bool packed = false;
        if (e == cudaSuccess && nchunk > 1) {
            e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
            for (int c = 0; c <= nchunk && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&pev[c], cudaEventDisableTiming);
            auto zc = [&](int c) { return (int)((long long)p->nz * c / nchunk); };
            for (int c = 0; c < nchunk && e == cudaSuccess; ++c) {
                const long long o = zc(c) * uplane, n = (zc(c + 1) - zc(c)) * uplane;
                e = cudaMemcpyAsync(dF + o, F + o, (size_t)n * 8, cudaMemcpyHostToDevice, h->wstream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(dO + o, omega + o, (size_t)n * 8, cudaMemcpyHostToDevice, h->wstream);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h->solid + o, solid + o, (size_t)n, cudaMemcpyHostToDevice, h->wstream);
                if (e == cudaSuccess) e = cudaEventRecord(pev[c], h->wstream);
            }
            // chunk c waits for chunk c + 1 (its upper neighbour plane); with a
            // periodic z the first and last chunks wait for the last one, and
            // the first goes last on the pack stream
            const bool wrap = p->periodic[2] != 0;
            for (int i = 0; i < nchunk && e == cudaSuccess; ++i) {
                const int c = wrap ? (i + 1) % nchunk : i;
                const int need = (wrap && (c == 0 || c == nchunk - 1)) ? nchunk - 1 : std::min(c + 1, nchunk - 1);
                e = cudaStreamWaitEvent(ps, pev[need], 0);
                if (e == cudaSuccess)
                    e = launch_pack(pv, p->weight_dtype, dF, dO, h->solid, p->alpha, nullptr, p->dt, p->kT, rf, ps,
                                    zc(c), zc(c + 1));
            }
            if (e == cudaSuccess) e = cudaEventRecord(pev[nchunk], ps);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->wstream, pev[nchunk], 0);
            packed = e == cudaSuccess;
        } else {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dF, F, (size_t)N * 8, cudaMemcpyHostToDevice, h->wstream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dO, omega, (size_t)N * 8, cudaMemcpyHostToDevice, h->wstream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->solid, solid, (size_t)N, cudaMemcpyHostToDevice, h->wstream);
        }
        if (e == cudaSuccess && rho0) e = cudaMemcpyAsync(dR0, rho0, (size_t)N * 8, cudaMemcpyHostToDevice, h->wstream);
        if (e == cudaSuccess && alpha_links) e = cudaMemcpyAsync(dA, alpha_links, (size_t)N * 24, cudaMemcpyHostToDevice, h->wstream);
        if (e == cudaSuccess && o.region) {
            // labels into rows of pitch Xr (0 in the row padding)
            e = cudaMemsetAsync(h->region, 0, region_bytes, h->wstream);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(h->region, (size_t)h->Xr, o.region, (size_t)p->nx, (size_t)p->nx,
                                      (size_t)p->ny * p->nz, cudaMemcpyHostToDevice, h->wstream);
        }
        // the byte mask is stored as given; solid means nonzero
        if (e == cudaSuccess && device_check)
            e = launch_check_inputs(dF, dO, h->solid, dR0, dA, N, h->counter + kInputCheckWord, h->wstream);
        if (e == cudaSuccess) st = ensure_history(h, 1024);
        if (e == cudaSuccess && st == LPC_OK) {
            LatticeView v = make_view(h, 1);   // writes go to buffer 0
            if (!packed)
                e = launch_pack(v, p->weight_dtype, dF, dO, h->solid, p->alpha, dA, p->dt, p->kT, rf, h->wstream);
            if (e == cudaSuccess)
                e = launch_init_state(v, dR0, p->init, dF, h->solid, p->kT, h->scratch, h->wstream);
            if (e == cudaSuccess) e = launch_reservoir_ghosts(v, rf, h->wstream);
            h->cur = 0;
            if (e == cudaSuccess) e = launch_sum_state(updated_view(h, 0), h->wstream);
            if (e == cudaSuccess)
                e = launch_region_sums(updated_view(h, 0), p->weight_dtype, h->rpart, h->counter + 12, false, h->wstream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
        if (ps) {
            // after an error the pack stream may still run: wait for it before the temporaries go
            cudaStreamSynchronize(ps);
            cudaStreamDestroy(ps);
        }
        for (int c = 0; c < 9; ++c)
            if (pev[c]) cudaEventDestroy(pev[c]);
    }
    dfree(h, dF, (size_t)N * 8); dfree(h, dO, (size_t)N * 8); dfree(h, dR0, (size_t)N * 8);
    dfree(h, dA, (size_t)N * 24);
    if (e == cudaSuccess && st == LPC_OK && device_check) {
        unsigned int bits = 0;
        e = cudaMemcpy(&bits, h->counter + kInputCheckWord, 4, cudaMemcpyDeviceToHost);
        const char* bad = (bits & 1u) ? "lattice_create: non-finite F on a pore site"
                        : (bits & 2u) ? "lattice_create: non-finite omega"
                        : (bits & 4u) ? "lattice_create: non-finite rho0 on a pore site"
                        : (bits & 8u) ? "lattice_create_links: link factors must be in [0, 1]" : nullptr;
        if (e == cudaSuccess && bad) {
            release_all(h); delete h;
            set_error(bad);
            return LPC_ERR_INVALID;
        }
    }
    if (e != cudaSuccess || st != LPC_OK) {
        if (st == LPC_OK) st = cuda_fail(e, "lattice_create");
        release_all(h); delete h;
        return st;
    }
    h->steps = 0;
    auto_schedule(h);
    *out = h;
    return LPC_OK;
}

// A whole lattice with a reservoir on a z face: the reservoir sites are a
// halo plane below (face 4) or above (face 5) the own planes, with free
// energy F_res and no solid; the hop weights between it and the boundary
// plane are then packed by the same Metropolis rule as every other link,
// which is the reservoir rule (reservoir links take the scalar alpha), and
// its state is set to the reservoir's values after the start state.  A z
// face without a reservoir gets an all-solid halo plane (a wall).  The
// fields are extended on the host (transient copies); the caller's arrays
// hold the nz own planes.
lpc_status create_with_z_halos(const lpc_params* p, const lpc_options& o, const double* F, const double* omega,
                               const uint8_t* solid, const double* rho0, const lpc_allocator* a, void* stream,
                               lpc_lattice** out) {
    const size_t plane = (size_t)p->nx * p->ny, N = plane * p->nz, N2 = plane * ((size_t)p->nz + 2);
    std::vector<double> F2, O2, R2, A2;
    std::vector<uint8_t> S2, L2;
    try {
        F2.assign(N2, 0.0);
        O2.assign(N2, 0.0);
        S2.assign(N2, 0);
        if (rho0) R2.assign(N2, 0.0);
        if (o.alpha_links) A2.assign(3 * N2, p->alpha);
        if (o.region) L2.assign(N2, 0);
    } catch (const std::bad_alloc&) {
        set_error("lattice_create_ex: host allocation failed (z reservoir planes)");
        return LPC_ERR_OOM;
    }
    memcpy(F2.data() + plane, F, N * 8);
    memcpy(O2.data() + plane, omega, N * 8);
    memcpy(S2.data() + plane, solid, N);
    if (rho0) memcpy(R2.data() + plane, rho0, N * 8);
    for (int ax = 0; ax < 3 && o.alpha_links; ++ax) memcpy(A2.data() + ax * N2 + plane, o.alpha_links + ax * N, N * 8);
    // the +z links of the last own plane end in the upper halo: a reservoir
    // link takes the scalar alpha (the caller's value there is unused)
    if (o.alpha_links)
        for (size_t i = 0; i < plane; ++i) A2[2 * N2 + plane * (size_t)p->nz + i] = p->alpha;
    if (o.region) memcpy(L2.data() + plane, o.region, N);
    for (int side = 0; side < 2; ++side) {
        const lpc_reservoir& r = o.reservoir[4 + side];
        const size_t z0 = side ? plane * ((size_t)p->nz + 1) : 0;
        for (size_t i = 0; i < plane; ++i) {
            F2[z0 + i] = r.enabled ? r.F : 0.0;
            S2[z0 + i] = r.enabled ? 0 : 1;
            if (rho0) R2[z0 + i] = r.enabled ? r.rho : 0.0;
        }
    }
    lpc_params q = *p;
    q.nz = p->nz + 2;
    lpc_options o2 = o;
    o2.alpha_links = o.alpha_links ? A2.data() : nullptr;
    o2.region = o.region ? L2.data() : nullptr;
    return create_impl(&q, &o2, F2.data(), O2.data(), S2.data(), rho0 ? R2.data() : nullptr, a, stream, out,
                       kZHalos);
}

}  // namespace

extern "C" {

lpc_status lattice_create_ex(const lpc_params* p, const lpc_options* opt, const double* F,
                             const double* omega, const uint8_t* solid, const double* rho0,
                             const lpc_allocator* a, void* stream, lpc_lattice** out) {
    return create_impl(p, opt, F, omega, solid, rho0, a, stream, out, kWhole);
}

lpc_status lattice_create_slab(const lpc_params* p, int32_t halo, const lpc_options* opt, const double* F,
                               const double* omega, const uint8_t* solid, const double* rho0,
                               const lpc_allocator* a, void* stream, lpc_lattice** out) {
    if (out) *out = nullptr;
    if (!p) { set_error("lattice_create_slab: NULL argument"); return LPC_ERR_INVALID; }
    if (halo != 1) { set_error("lattice_create_slab: halo must be 1 (one plane on each side)"); return LPC_ERR_INVALID; }
    if (p->nz < 1 || p->nz > 2147483647 - 2) { set_error("lattice_create_slab: edges must be >= 1"); return LPC_ERR_INVALID; }
    lpc_params q = *p;
    q.nz = p->nz + 2;          // the halo planes below and above the slab's own planes
    q.periodic[2] = 0;         // the halos bound the slab: no plane index wraps
    return create_impl(&q, opt, F, omega, solid, rho0, a, stream, out, kSlab);
}

lpc_status lattice_slab_planes(lpc_lattice* h, int32_t which, lpc_plane_set* out) {
    if (!h || !out) { set_error("lattice_slab_planes: NULL argument"); return LPC_ERR_INVALID; }
    if (!h->slab) { set_error("lattice_slab_planes: not a slab (lattice_create_slab)"); return LPC_ERR_INVALID; }
    if (which < 0 || which > 3) { set_error("lattice_slab_planes: which must be 0..3"); return LPC_ERR_INVALID; }
    const int z = which == LPC_PLANE_FIRST ? h->zlo
                : which == LPC_PLANE_LAST ? h->zhi - 1
                : which == LPC_PLANE_HALO_BELOW ? h->zlo - 1 : h->zhi;
    const long long plane = (long long)h->Xp * h->Yp;
    const long long off = (long long)z * plane;
    memset(out, 0, sizeof *out);
    out->plane[0] = h->rho[h->cur] + off;
    out->bytes[0] = plane * 4;
    out->plane[1] = h->m[h->cur] + off;
    out->bytes[1] = plane * 8;
    for (int a = 0; a < 3; ++a)
        if (h->mu[h->cur][a]) {
            out->plane[2 + a] = h->mu[h->cur][a] + off;
            out->bytes[2 + a] = plane * 4;
        }
    return LPC_OK;
}

lpc_status lattice_footprint(const lpc_params* p, int64_t steps, int64_t* bytes) {
    if (!p || !bytes || steps < 0) { set_error("lattice_footprint: bad arguments"); return LPC_ERR_INVALID; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->ghost < 0 || p->ghost > kMaxGhost || (p->ghost & 1) ||
        p->msd_axes < 0 || p->msd_axes > 7) {
        set_error("lattice_footprint: bad parameters");
        return LPC_ERR_INVALID;
    }
    const long long N = (long long)p->nx * p->ny * p->nz;
    int G = p->ghost;
    if (G == 0) G = 2;
    const long long Xp = ((p->nx + 2 * G) + 31) / 32 * 32, Yp = p->ny + 2 * G;
    const long long Np = Xp * Yp * p->nz;
    int na = 0;
    for (int a = 0; a < 3; ++a) na += p->msd_axes >> a & 1;
    const long long wb = p->weight_dtype == LPC_WEIGHTS_BF16 ? 2 : 4;
    long long cap = steps + 1 < 1024 ? 1024 : steps + 1;
    long long b = Np * (2 * 4 + 2 * 8 + 2 * 4 * na + 6 * wb + 8) + N;
    b += (long long)device_props().sm_count * 32 * kMaxTB * kNumSums * 8 + 256 + 8 * 1024;
    b += (long long)history_bytes(cap, 1);
    b += 16 * N;    // transient copies of F and omega during create
    if (p->nx >= 64 && p->ny >= 16 && N >= (1LL << 20))     // the automatic schedule's gather form
        b += (long long)gather_bytes((long long)gather_pitch(p->nx) * p->ny * p->nz, *p, 0);
    *bytes = b;
    return LPC_OK;
}

lpc_status lattice_destroy(lpc_lattice* h) {
    if (!h) return LPC_OK;
    cudaSetDevice(h->device);
    release_all(h);
    delete h;
    return LPC_OK;
}

lpc_status lattice_set_schedule(lpc_lattice* h, int32_t kernel, int32_t block_steps) {
    if (!h) { set_error("lattice_set_schedule: NULL handle"); return LPC_ERR_INVALID; }
    if (kernel == LPC_KERNEL_AUTO) {
        auto_schedule(h);
        return LPC_OK;
    }
    if (kernel == LPC_KERNEL_STEP1) {
        h->kernel = LPC_KERNEL_STEP1; h->kdepth = 1;
        drop_graphs(h);
        return LPC_OK;
    }
    if (kernel == LPC_KERNEL_TB) {
        cudaSetDevice(h->device);
        int bw = 0, bh = 0;
        if (!tb_supported(make_view(h, 0), h->p.weight_dtype, block_steps) ||
            !tb_box_dims(make_view(h, 0), h->p.weight_dtype, block_steps, &bw, &bh)) {
            set_error("lattice_set_schedule: TB needs 1 <= block_steps <= min(4, ghost)");
            return LPC_ERR_INVALID;
        }
        if (!tb_depth_allowed(h, block_steps)) {
            set_error("lattice_set_schedule: lattices with reservoirs or regions take one step per launch");
            return LPC_ERR_INVALID;
        }
        cudaError_t e = tb_prepare(h->p.weight_dtype, block_steps, h->p.msd_axes);
        if (e != cudaSuccess) return cuda_fail(e, "lattice_set_schedule");
        h->kernel = LPC_KERNEL_TB;
        h->kdepth = block_steps;
        drop_graphs(h);
        return LPC_OK;
    }
    set_error("lattice_set_schedule: unknown kernel");
    return LPC_ERR_INVALID;
}

lpc_status lattice_set_static_form(lpc_lattice* h, int32_t form) {
    if (!h) { set_error("lattice_set_static_form: NULL handle"); return LPC_ERR_INVALID; }
    if (form != LPC_STATIC_AUTO && form != LPC_STATIC_GATHER && form != LPC_STATIC_LINK) {
        set_error("lattice_set_static_form: form must be LPC_STATIC_AUTO, _GATHER or _LINK");
        return LPC_ERR_INVALID;
    }
    if (form == LPC_STATIC_LINK && !link_form_possible(h)) {
        set_error("lattice_set_static_form: the link form needs one jump factor, no reservoir face and no regions");
        return LPC_ERR_INVALID;
    }
    cudaSetDevice(h->device);
    Entry en(h);
    h->static_pref = form;
    drop_static(h);
    // made now when the one-step TMA kernel is the lattice's schedule (so a
    // failure is reported here), else on that kernel's first launch
    if (h->kernel == LPC_KERNEL_TB && h->kdepth == 1) {
        const lpc_status st = ensure_maps(h);
        if (st != LPC_OK) return st;
    }
    return LPC_OK;
}

lpc_status lattice_set_tiling(lpc_lattice* h, int32_t tile_rows, int32_t items_per_cta) {
    if (!h) { set_error("lattice_set_tiling: NULL handle"); return LPC_ERR_INVALID; }
    if (tile_rows != 0 && tile_rows != 8 && tile_rows != 12 && tile_rows != 16) {
        set_error("lattice_set_tiling: tile_rows must be 0 (heuristic), 8, 12 or 16");
        return LPC_ERR_INVALID;
    }
    if (items_per_cta != 0 && (items_per_cta < 1 || items_per_cta > 1024)) {
        set_error("lattice_set_tiling: items_per_cta must be 0 (heuristic) or 1..1024");
        return LPC_ERR_INVALID;
    }
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->wstream);
    h->t1_ty = tile_rows;
    h->t1_ipc = items_per_cta;
    h->maps_K = 0;
    drop_graphs(h);
    return LPC_OK;
}

lpc_status lattice_step_n(lpc_lattice* h, int64_t n) {
    Range nvtx("lattice_step_n");
    if (!h) { set_error("lattice_step_n: NULL handle"); return LPC_ERR_INVALID; }
    if (n < 0) { set_error("lattice_step_n: n must be >= 0"); return LPC_ERR_INVALID; }
    if (n == 0) return LPC_OK;
    Entry en(h);
    lpc_status st = ensure_history(h, h->steps + n + 1);
    if (st != LPC_OK) return st;
    const bool tb = h->kernel == LPC_KERNEL_TB;
    const long long per = tb ? h->kdepth : 1;     // steps per launch
    long long launches = n / per;
    long long rest = n % per;                    // remainder: one-step launches
    while (launches >= kGraphLen) {
        if (!h->graph[h->cur]) {
            st = build_graph(h, h->cur);
            if (st != LPC_OK) return st;
        }
        cudaError_t e = cudaGraphLaunch(h->graph[h->cur], h->wstream);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        launches -= kGraphLen;     // kGraphLen is even: parity unchanged
    }
    for (; launches > 0; --launches) {
        st = launch_one(h, h->wstream, tb);
        if (st != LPC_OK) return st;
    }
    for (; rest > 0; --rest) {
        st = launch_one(h, h->wstream, false);
        if (st != LPC_OK) return st;
    }
    h->steps += n;
    return LPC_OK;
}

lpc_status lattice_step_many(lpc_lattice* const* hs, const int64_t* n, int32_t count) {
    Range nvtx("lattice_step_many");
    if (count < 0 || (count > 0 && (!hs || !n))) { set_error("lattice_step_many: bad arguments"); return LPC_ERR_INVALID; }
    if (count == 0) return LPC_OK;
    long long max_n = 0;
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || n[i] < 0) { set_error("lattice_step_many: NULL handle or negative step count"); return LPC_ERR_INVALID; }
        if (hs[i]->device != hs[0]->device) { set_error("lattice_step_many: lattices on different devices"); return LPC_ERR_INVALID; }
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) { set_error("lattice_step_many: a lattice appears twice"); return LPC_ERR_INVALID; }
        if (n[i] > max_n) max_n = n[i];
    }
    lpc_lattice* h0 = hs[0];
    cudaSetDevice(h0->device);
    cudaStream_t bs = h0->wstream;
    // order the batch stream after every lattice's caller stream
    for (int i = 0; i < count; ++i) {
        lpc_status st = ensure_history(hs[i], hs[i]->steps + n[i] + 1);
        if (st != LPC_OK) return st;
        cudaEventRecord(hs[i]->ev_in, hs[i]->ustream);
        cudaStreamWaitEvent(bs, hs[i]->ev_in, 0);
        cudaEventRecord(hs[i]->ev_in, hs[i]->wstream);
        cudaStreamWaitEvent(bs, hs[i]->ev_in, 0);
    }
    // lattices on the TMA-fed one-step kernel share multi-lattice launches
    // (per group of weight type, tile height and ghost width); the others
    // are batched with the register-pipelined kernel, or step alone where
    // their item partials do not fit their buffer
    std::vector<int> alone;
    std::vector<int> batched;
    std::vector<int> multi;
    lpc_status status = LPC_OK;
    for (int i = 0; i < count && status == LPC_OK; ++i) {
        lpc_lattice* h = hs[i];
        if (n[i] > 0 && h->kernel == LPC_KERNEL_TB && h->kdepth == 1) {
            status = ensure_maps(h);        // static data and tensor maps, outside the launches
            if (status == LPC_OK && t1_multi_member(make_view(h, h->cur), h->p.weight_dtype)) {
                multi.push_back(i);
                continue;
            }
        }
        int tx, ty, cz;
        const int items = batch_items(make_view(h, h->cur), &tx, &ty, &cz);
        if ((size_t)items * kNumSums > h->partials_doubles || h->nreg > 0 || h->zlo > 0) alone.push_back(i);
        else batched.push_back(i);
    }
    if (status != LPC_OK) return status;
    static thread_local BatchParams bp;
    // multi-lattice TMA launches: one per step and group chunk, over the
    // lattices with steps left (sorted by step count, so they form a prefix)
    {
        std::vector<int> order = multi;
        std::vector<int> key(count, 0);
        for (int i : multi) key[i] = t1_multi_group(make_view(hs[i], hs[i]->cur), hs[i]->p.weight_dtype);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return key[a] != key[b] ? key[a] < key[b] : n[a] > n[b]; });
        static thread_local std::vector<LatticeView> views;
        static thread_local std::vector<const TBMaps*> mps;
        for (size_t g0 = 0; g0 < order.size() && status == LPC_OK;) {
            size_t g1 = g0;
            while (g1 < order.size() && key[order[g1]] == key[order[g0]]) ++g1;
            const int wd = hs[order[g0]]->p.weight_dtype;
            for (size_t c0 = g0; c0 < g1 && status == LPC_OK; c0 += kMaxMulti) {
                const size_t c1 = std::min(g1, c0 + (size_t)kMaxMulti);
                const long long steps_c = n[order[c0]];
                for (long long s = 0; s < steps_c && status == LPC_OK; ++s) {
                    views.clear();
                    mps.clear();
                    for (size_t j = c0; j < c1; ++j) {
                        lpc_lattice* h = hs[order[j]];
                        if (n[order[j]] <= s) break;          // sorted: the rest are done too
                        views.push_back(make_view(h, h->cur));
                        mps.push_back(h->maps[h->cur]);
                    }
                    const cudaError_t e = launch_tma1_multi(views.data(), mps.data(), (int)views.size(), wd,
                                                            h0->counter + 20, bs);
                    if (e != cudaSuccess) { status = cuda_fail(e, "multi-lattice step launch"); break; }
                    for (size_t j = 0; j < views.size(); ++j) hs[order[c0 + j]]->cur ^= 1;
                }
            }
            g0 = g1;
        }
    }
    // per (weight type, MSD mask) group, chunks of kMaxBatch lattices sorted
    // by step count: one persistent launch runs every step of a chunk; where
    // a cooperative launch is not possible, one launch per step
    for (int wd = 0; wd < 2 && status == LPC_OK; ++wd)
        for (int msd = 0; msd < 8 && status == LPC_OK; ++msd) {
            std::vector<int> group;
            for (int i : batched)
                if (n[i] > 0 && hs[i]->p.weight_dtype == wd && hs[i]->p.msd_axes == msd) group.push_back(i);
            std::stable_sort(group.begin(), group.end(), [&](int a, int b) { return n[a] > n[b]; });
            for (size_t c0 = 0; c0 < group.size() && status == LPC_OK; c0 += kMaxBatch) {
                const size_t c1 = std::min(group.size(), c0 + (size_t)kMaxBatch);
                bp.count = 0;
                bp.total_items = 0;
                for (size_t j = c0; j < c1; ++j) {
                    lpc_lattice* h = hs[group[j]];
                    BatchEntry& E = bp.e[bp.count++];
                    E.v = make_view(h, h->cur);
                    E.n_items = batch_items(E.v, &E.tiles_x, &E.tiles_y, &E.cz);
                    E.item0 = bp.total_items;
                    E.steps = (int)std::min<int64_t>(n[group[j]], INT32_MAX);
                    bp.total_items += E.n_items;
                }
                const long long steps_c = n[group[c0]];
                cudaError_t e = steps_c <= INT32_MAX
                                    ? launch_batch_multi(bp, wd, msd, (int)steps_c, h0->counter + 9, bs)
                                    : cudaErrorInvalidValue;
                if (e == cudaSuccess) {
                    for (size_t j = c0; j < c1; ++j) hs[group[j]]->cur ^= (int)(n[group[j]] & 1);
                    continue;
                }
                cudaGetLastError();
                for (long long s = 0; s < steps_c && status == LPC_OK; ++s) {
                    bp.count = 0;
                    bp.total_items = 0;
                    for (size_t j = c0; j < c1; ++j) {
                        lpc_lattice* h = hs[group[j]];
                        if (n[group[j]] <= s) continue;
                        BatchEntry& E = bp.e[bp.count++];
                        E.v = make_view(h, h->cur);
                        E.n_items = batch_items(E.v, &E.tiles_x, &E.tiles_y, &E.cz);
                        E.item0 = bp.total_items;
                        E.steps = 1;
                        bp.total_items += E.n_items;
                        h->cur ^= 1;
                    }
                    const cudaError_t e1 = launch_batch(bp, wd, msd, bs);
                    if (e1 != cudaSuccess) status = cuda_fail(e1, "batched step launch");
                }
            }
        }
    for (int i : alone)
        for (long long s = 0; s < n[i] && status == LPC_OK; ++s)
            status = launch_one(hs[i], bs, hs[i]->kernel == LPC_KERNEL_TB && hs[i]->kdepth == 1);
    for (int i = 0; i < count; ++i) hs[i]->steps += n[i];
    // every lattice's private stream continues after the batch (queries and
    // later calls synchronise on it); callers' streams are left free so that
    // new lattices can be created while a batch runs
    cudaEventRecord(h0->ev_out, bs);
    for (int i = 0; i < count; ++i)
        if (hs[i]->wstream != bs) cudaStreamWaitEvent(hs[i]->wstream, h0->ev_out, 0);
    return status;
}

lpc_status lattice_autotune(lpc_lattice* h, int32_t trial_launches, int32_t* kernel, int32_t* block_steps,
                            double* rate) {
    Range nvtx("lattice_autotune");
    if (!h || trial_launches < 1) { set_error("lattice_autotune: bad arguments"); return LPC_ERR_INVALID; }
    Entry en(h);
    const size_t Np = (size_t)h->Np;
    int na = 0;
    for (int a = 0; a < 3; ++a) na += h->p.msd_axes >> a & 1;
    // snapshot of the current state (the trials advance it)
    const size_t snap_bytes = Np * (12 + 4 * (size_t)na);
    char* snap = (char*)dalloc(h, snap_bytes);
    if (!snap) { set_error("lattice_autotune: snapshot allocation failed"); return LPC_ERR_OOM; }
    const int cur0 = h->cur;
    const long long steps0 = h->steps;
    const int kernel0 = h->kernel, k0 = h->kdepth;
    cudaError_t e = cudaMemcpyAsync(snap, h->rho[cur0], Np * 4, cudaMemcpyDeviceToDevice, h->wstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap + Np * 4, h->m[cur0], Np * 8, cudaMemcpyDeviceToDevice, h->wstream);
    for (int a = 0, n = 0; a < 3 && e == cudaSuccess; ++a)
        if (h->p.msd_axes >> a & 1)
            e = cudaMemcpyAsync(snap + Np * (12 + 4 * (size_t)n++), h->mu[cur0][a], Np * 4, cudaMemcpyDeviceToDevice, h->wstream);
    if (e != cudaSuccess) { dfree(h, snap, snap_bytes); return cuda_fail(e, "lattice_autotune: snapshot"); }
    // the trials write history entries after steps0; make room for them
    const int maxk = h->G < 4 ? h->G : 4;
    lpc_status st = ensure_history(h, steps0 + (long long)(trial_launches + 2) * maxk + 2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // candidates: the register-pipelined kernel; the TMA-fed one-step kernel
    // at every tile height and three work-item sizes; TB at depth 2..maxk
    struct Cand { int kernel, K, ty, ipc; };
    std::vector<Cand> cands{{LPC_KERNEL_STEP1, 1, 0, 0}};
    for (int ty : {16, 12, 8})
        for (int ipc : {20, 40, 80}) cands.push_back({LPC_KERNEL_TB, 1, ty, ipc});
    for (int K = 2; K <= maxk; ++K) cands.push_back({LPC_KERNEL_TB, K, 0, 0});
    const int ty0 = h->t1_ty, ipc0 = h->t1_ipc;
    Cand best_c{LPC_KERNEL_STEP1, 1, 0, 0};
    double best = -1.0;
    for (const Cand& c : cands) {
        if (st != LPC_OK) break;
        const bool tb = c.kernel == LPC_KERNEL_TB;
        const int K = c.K;
        if (tb && (!tb_supported(make_view(h, 0), h->p.weight_dtype, K) || !tb_depth_allowed(h, K))) continue;
        if (tb) {
            h->kernel = LPC_KERNEL_TB;
            h->kdepth = K;
            h->t1_ty = c.ty;
            h->t1_ipc = c.ipc;
            h->maps_K = 0;                 // re-encode the tensor maps for this tiling
            if (tb_prepare(h->p.weight_dtype, K, h->p.msd_axes) != cudaSuccess) continue;
            if (K == 1) {
                st = ensure_maps(h);          // static data and tensor maps for this tiling
                if (st != LPC_OK) break;
                // a tile height the rings cannot hold falls back to the heuristic: skip it
                if (t1_tile_rows(make_view(h, 0), h->p.weight_dtype) != c.ty) continue;
            }
        } else {
            h->kernel = LPC_KERNEL_STEP1;
            h->kdepth = 1;
        }
        for (int i = 0; i < 2 && st == LPC_OK; ++i) st = launch_one(h, h->wstream, tb);
        cudaEventRecord(e0, h->wstream);
        for (int i = 0; i < trial_launches && st == LPC_OK; ++i) st = launch_one(h, h->wstream, tb);
        cudaEventRecord(e1, h->wstream);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(e, "lattice_autotune: trial"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double r = (double)n_updated(h) * K * trial_launches / (ms * 1e-3);
        if (r > best) { best = r; best_c = c; }
        // the device step counter advanced; put it back for the next trial
        const long long s0 = steps0;
        cudaMemcpyAsync(h->dstep, &s0, 8, cudaMemcpyHostToDevice, h->wstream);
        cudaStreamSynchronize(h->wstream);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the state into the buffer that was current
    h->cur = cur0;
    e = cudaMemcpyAsync(h->rho[cur0], snap, Np * 4, cudaMemcpyDeviceToDevice, h->wstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->m[cur0], snap + Np * 4, Np * 8, cudaMemcpyDeviceToDevice, h->wstream);
    for (int a = 0, n = 0; a < 3 && e == cudaSuccess; ++a)
        if (h->p.msd_axes >> a & 1)
            e = cudaMemcpyAsync(h->mu[cur0][a], snap + Np * (12 + 4 * (size_t)n++), Np * 4, cudaMemcpyDeviceToDevice, h->wstream);
    const long long s0 = steps0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dstep, &s0, 8, cudaMemcpyHostToDevice, h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    dfree(h, snap, snap_bytes);
    h->steps = steps0;
    if (st != LPC_OK) {
        h->kernel = kernel0; h->kdepth = k0; h->t1_ty = ty0; h->t1_ipc = ipc0; h->maps_K = 0;
        drop_graphs(h);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "lattice_autotune: restore");
    h->kernel = best_c.kernel;
    h->kdepth = best_c.K;
    h->t1_ty = best_c.ty;
    h->t1_ipc = best_c.ipc;
    h->maps_K = 0;
    drop_graphs(h);
    if (kernel) *kernel = best_c.kernel;
    if (block_steps) *block_steps = best_c.K;
    if (rate) *rate = best;
    return LPC_OK;
}

lpc_status lattice_sync(lpc_lattice* h) {
    if (!h) { set_error("lattice_sync: NULL handle"); return LPC_ERR_INVALID; }
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->ustream);
    if (e != cudaSuccess) return cuda_fail(e, "lattice_sync");
    return check_device_error(h);
}

lpc_status lattice_steps_done(lpc_lattice* h, int64_t* n) {
    if (!h || !n) { set_error("lattice_steps_done: NULL argument"); return LPC_ERR_INVALID; }
    *n = h->steps;
    return LPC_OK;
}

lpc_status lattice_info(lpc_lattice* h, lpc_info* out) {
    if (!h || !out) { set_error("lattice_info: NULL argument"); return LPC_ERR_INVALID; }
    out->n_sites = n_updated(h);
    out->n_padded = h->Np;
    out->ghost = h->G;
    out->pitch_x = h->Xp;
    out->pitch_y = h->Yp;
    out->kernel = h->kernel;
    out->block_steps = h->kdepth;
    out->static_form = h->lnk ? 2 : (h->gwin ? 1 : 0);
    out->tile_rows = t1_tile_rows(make_view(h, h->cur), h->p.weight_dtype);
    out->items_per_cta = h->t1_ipc > 0 ? h->t1_ipc : t1_default_items_per_cta();
    out->device_bytes = h->device_bytes;
    long long b = 24 + 6 * (long long)wbytes(h) + 8;
    for (int a = 0; a < 3; ++a) if (h->p.msd_axes >> a & 1) b += 8;
    if (h->nreg > 0) b += 1;      // the region label of the site
    out->bytes_per_site_update = b;
    return LPC_OK;
}

static lpc_status range_check(lpc_lattice* h, int64_t first, int64_t count, const void* out, const char* who) {
    if (!h || (!out && count > 0)) { set_error(std::string(who) + ": NULL argument"); return LPC_ERR_INVALID; }
    if (first < 0 || count < 0 || first + count > h->steps + 1) {
        set_error(std::string(who) + ": range outside 0..steps_done");
        return LPC_ERR_INVALID;
    }
    return LPC_OK;
}

lpc_status lattice_fid(lpc_lattice* h, int64_t first, int64_t count, double* out) {
    lpc_status s = range_check(h, first, count, out, "lattice_fid");
    if (s != LPC_OK || count == 0) return s;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) { lpc_status ds = check_device_error(h); if (ds != LPC_OK) return ds; }
    if (e == cudaSuccess) e = cudaMemcpy(out, h->histM + first, sizeof(double2) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_fid");
}

lpc_status lattice_population(lpc_lattice* h, int64_t first, int64_t count, double* out) {
    lpc_status s = range_check(h, first, count, out, "lattice_population");
    if (s != LPC_OK || count == 0) return s;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) e = cudaMemcpy(out, h->histP + first, sizeof(double) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_population");
}

lpc_status lattice_msd(lpc_lattice* h, int32_t axis, int64_t first, int64_t count, double* out) {
    lpc_status s = range_check(h, first, count, out, "lattice_msd");
    if (s != LPC_OK) return s;
    if (axis < 0 || axis > 2 || !(h->p.msd_axes >> axis & 1)) { set_error("lattice_msd: axis not enabled"); return LPC_ERR_INVALID; }
    if (count == 0) return LPC_OK;
    cudaSetDevice(h->device);
    const long long upto = first + count - 1;   // need dMSD[0 .. upto-1]
    std::vector<double> d((size_t)(upto > 0 ? upto : 1));
    double P0 = 0.0;
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess && upto > 0) e = cudaMemcpy(d.data(), h->histD + axis * h->cap, sizeof(double) * upto, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&P0, h->histP, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "lattice_msd");
    double acc = 0.0;
    for (long long n = 0; n <= upto; ++n) {
        if (n >= first) out[n - first] = acc / P0;
        if (n < upto) acc += d[(size_t)n];
    }
    return LPC_OK;
}

lpc_status lattice_dmsd(lpc_lattice* h, int32_t axis, int64_t first, int64_t count, double* out) {
    if (!h || (!out && count > 0)) { set_error("lattice_dmsd: NULL argument"); return LPC_ERR_INVALID; }
    if (first < 0 || count < 0 || first + count > h->steps) { set_error("lattice_dmsd: range outside 0..steps_done-1"); return LPC_ERR_INVALID; }
    if (axis < 0 || axis > 2 || !(h->p.msd_axes >> axis & 1)) { set_error("lattice_dmsd: axis not enabled"); return LPC_ERR_INVALID; }
    if (count == 0) return LPC_OK;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) { lpc_status ds = check_device_error(h); if (ds != LPC_OK) return ds; }
    if (e == cudaSuccess)
        e = cudaMemcpy(out, h->histD + axis * h->cap + first, sizeof(double) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_dmsd");
}

static lpc_status region_check(lpc_lattice* h, int32_t region, const char* who) {
    if (!h) { set_error(std::string(who) + ": NULL handle"); return LPC_ERR_INVALID; }
    if (h->nreg == 0 || region < 0 || region >= h->nreg) {
        set_error(std::string(who) + ": region outside 0..n_regions-1 (or no regions)");
        return LPC_ERR_INVALID;
    }
    return LPC_OK;
}

lpc_status lattice_fid_region(lpc_lattice* h, int32_t region, int64_t first, int64_t count, double* out) {
    lpc_status s = region_check(h, region, "lattice_fid_region");
    if (s == LPC_OK) s = range_check(h, first, count, out, "lattice_fid_region");
    if (s != LPC_OK || count == 0) return s;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) { lpc_status ds = check_device_error(h); if (ds != LPC_OK) return ds; }
    if (e == cudaSuccess)
        e = cudaMemcpy(out, h->histM + (1 + region) * h->cap + first, sizeof(double2) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_fid_region");
}

lpc_status lattice_population_region(lpc_lattice* h, int32_t region, int64_t first, int64_t count,
                                     double* out) {
    lpc_status s = region_check(h, region, "lattice_population_region");
    if (s == LPC_OK) s = range_check(h, first, count, out, "lattice_population_region");
    if (s != LPC_OK || count == 0) return s;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, h->histP + (1 + region) * h->cap + first, sizeof(double) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_population_region");
}

lpc_status lattice_msd_region(lpc_lattice* h, int32_t region, int32_t axis, int64_t first, int64_t count,
                              double* out) {
    lpc_status s = region_check(h, region, "lattice_msd_region");
    if (s == LPC_OK) s = range_check(h, first, count, out, "lattice_msd_region");
    if (s != LPC_OK) return s;
    if (axis < 0 || axis > 2 || !(h->p.msd_axes >> axis & 1)) { set_error("lattice_msd_region: axis not enabled"); return LPC_ERR_INVALID; }
    if (count == 0) return LPC_OK;
    cudaSetDevice(h->device);
    const long long upto = first + count - 1;
    std::vector<double> d((size_t)(upto > 0 ? upto : 1));
    double P0 = 0.0;
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess && upto > 0)
        e = cudaMemcpy(d.data(), h->histD + ((1 + region) * 3 + axis) * h->cap, sizeof(double) * upto,
                       cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&P0, h->histP, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "lattice_msd_region");
    double acc = 0.0;
    for (long long n = 0; n <= upto; ++n) {
        if (n >= first) out[n - first] = acc / P0;
        if (n < upto) acc += d[(size_t)n];
    }
    return LPC_OK;
}

// Interior sites of a padded field into `out` (C order): a slab's own planes
// (all_planes = false) or every plane, halos included (checkpoints).
static lpc_status read_field(lpc_lattice* h, const void* src, int elem, void* out, int32_t out_is_device, const char* who,
                             bool all_planes = false) {
    if (!h || !out) { set_error(std::string(who) + ": NULL argument"); return LPC_ERR_INVALID; }
    Entry en(h);
    LatticeView v = make_view(h, h->cur);
    size_t n = (size_t)h->N;
    if (!all_planes && h->zlo > 0) {
        v.nz = h->zhi - h->zlo;
        src = static_cast<const char*>(src) + (size_t)h->zlo * h->Xp * h->Yp * elem;
        n = (size_t)n_updated(h);
    }
    void* dst = out;
    void* tmp = nullptr;
    if (!out_is_device) {
        tmp = dalloc(h, n * elem);
        if (!tmp) { set_error(std::string(who) + ": temporary allocation failed"); return LPC_ERR_OOM; }
        dst = tmp;
    }
    cudaError_t e = launch_unpad(src, elem, v, dst, h->wstream);
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, n * elem, cudaMemcpyDeviceToHost, h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    if (tmp) dfree(h, tmp, n * elem);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, who);
}

lpc_status lattice_density(lpc_lattice* h, float* out, int32_t out_is_device) {
    Range nvtx("lattice_density");
    if (!h) { set_error("lattice_density: NULL handle"); return LPC_ERR_INVALID; }
    return read_field(h, h->rho[h->cur], 4, out, out_is_device, "lattice_density");
}

lpc_status lattice_magnetization(lpc_lattice* h, float* out, int32_t out_is_device) {
    if (!h) { set_error("lattice_magnetization: NULL handle"); return LPC_ERR_INVALID; }
    return read_field(h, h->m[h->cur], 8, out, out_is_device, "lattice_magnetization");
}

lpc_status lattice_moment(lpc_lattice* h, int32_t axis, float* out, int32_t out_is_device) {
    if (!h) { set_error("lattice_moment: NULL handle"); return LPC_ERR_INVALID; }
    if (axis < 0 || axis > 2 || !(h->p.msd_axes >> axis & 1)) { set_error("lattice_moment: axis not enabled"); return LPC_ERR_INVALID; }
    return read_field(h, h->mu[h->cur][axis], 4, out, out_is_device, "lattice_moment");
}

lpc_status lattice_weights(lpc_lattice* h, float* out) {
    if (!h || !out) { set_error("lattice_weights: NULL argument"); return LPC_ERR_INVALID; }
    Entry en(h);
    const size_t n = (size_t)n_updated(h);
    float* tmp = (float*)dalloc(h, n * 6 * 4);
    if (!tmp) { set_error("lattice_weights: temporary allocation failed"); return LPC_ERR_OOM; }
    cudaError_t e = launch_weights_f32(updated_view(h, h->cur), h->p.weight_dtype, tmp, h->wstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * 24, cudaMemcpyDeviceToHost, h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    dfree(h, tmp, n * 24);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_weights");
}

lpc_status lattice_rotation(lpc_lattice* h, float* out) {
    if (!h) { set_error("lattice_rotation: NULL handle"); return LPC_ERR_INVALID; }
    return read_field(h, h->R, 8, out, 0, "lattice_rotation");
}

lpc_status lattice_solid(lpc_lattice* h, uint8_t* out) {
    if (!h || !out) { set_error("lattice_solid: NULL argument"); return LPC_ERR_INVALID; }
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, h->solid + (size_t)h->zlo * h->p.nx * h->p.ny, (size_t)n_updated(h), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_solid");
}

// State blob: header, rho [N] f32, m [N] f32x2, mu [axes][N] f32, M [steps+1]
// f64x2, P [steps+1] f64, dMSD [axes][steps] f64.
struct StateHeader {
    char magic[8];
    int32_t nx, ny, nz, msd_axes;
    int64_t steps;
    int32_t n_regions, reserved;
};

static const char kStateMagic[9] = "LPC3DST2";

// header, state (rho, m, mu), then one history set (M, P, dMSD of the
// enabled axes) for the totals and one per region
static size_t state_bytes(const lpc_lattice* h) {
    int na = 0;
    for (int a = 0; a < 3; ++a) na += h->p.msd_axes >> a & 1;
    const size_t N = (size_t)h->N;
    const size_t S = (size_t)h->steps;
    return sizeof(StateHeader) + N * (12 + 4 * na) + (1 + (size_t)h->nreg) * ((S + 1) * 24 + S * 8 * na);
}

lpc_status lattice_state_size(lpc_lattice* h, size_t* bytes) {
    if (!h || !bytes) { set_error("lattice_state_size: NULL argument"); return LPC_ERR_INVALID; }
    *bytes = state_bytes(h);
    return LPC_OK;
}

lpc_status lattice_get_state(lpc_lattice* h, void* buf, size_t bytes) {
    Range nvtx("lattice_get_state");
    if (!h || !buf) { set_error("lattice_get_state: NULL argument"); return LPC_ERR_INVALID; }
    if (bytes < state_bytes(h)) { set_error("lattice_get_state: buffer too small"); return LPC_ERR_INVALID; }
    char* p = (char*)buf;
    StateHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, kStateMagic, 8);
    hd.nx = h->p.nx; hd.ny = h->p.ny; hd.nz = h->p.nz; hd.msd_axes = h->p.msd_axes; hd.steps = h->steps;
    hd.n_regions = h->nreg;
    memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t N = (size_t)h->N;
    lpc_status s = read_field(h, h->rho[h->cur], 4, p, 0, "lattice_get_state", true);
    if (s != LPC_OK) return s;
    p += N * 4;
    s = read_field(h, h->m[h->cur], 8, p, 0, "lattice_get_state", true);
    if (s != LPC_OK) return s;
    p += N * 8;
    for (int a = 0; a < 3; ++a) {
        if (!(h->p.msd_axes >> a & 1)) continue;
        s = read_field(h, h->mu[h->cur][a], 4, p, 0, "lattice_get_state", true);
        if (s != LPC_OK) return s;
        p += N * 4;
    }
    const size_t S = (size_t)h->steps;
    cudaError_t e = cudaSuccess;
    for (int set = 0; set <= h->nreg && e == cudaSuccess; ++set) {
        e = cudaMemcpy(p, h->histM + set * h->cap, (S + 1) * 16, cudaMemcpyDeviceToHost);
        p += (S + 1) * 16;
        if (e == cudaSuccess) e = cudaMemcpy(p, h->histP + set * h->cap, (S + 1) * 8, cudaMemcpyDeviceToHost);
        p += (S + 1) * 8;
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            if (!(h->p.msd_axes >> a & 1)) continue;
            if (S > 0) e = cudaMemcpy(p, h->histD + (set * 3 + a) * h->cap, S * 8, cudaMemcpyDeviceToHost);
            p += S * 8;
        }
    }
    return e == cudaSuccess ? LPC_OK : cuda_fail(e, "lattice_get_state");
}

lpc_status lattice_set_state(lpc_lattice* h, const void* buf, size_t bytes) {
    Range nvtx("lattice_set_state");
    if (!h || !buf) { set_error("lattice_set_state: NULL argument"); return LPC_ERR_INVALID; }
    if (bytes < sizeof(StateHeader)) { set_error("lattice_set_state: buffer too small"); return LPC_ERR_INVALID; }
    StateHeader hd;
    memcpy(&hd, buf, sizeof hd);
    if (memcmp(hd.magic, kStateMagic, 8) != 0 || hd.nx != h->p.nx || hd.ny != h->p.ny || hd.nz != h->p.nz ||
        hd.msd_axes != h->p.msd_axes || hd.steps < 0 || hd.n_regions != h->nreg) {
        set_error("lattice_set_state: blob does not match this lattice");
        return LPC_ERR_INVALID;
    }
    const long long old_steps = h->steps;
    h->steps = hd.steps;
    const size_t need = state_bytes(h);
    h->steps = old_steps;
    if (bytes < need) { set_error("lattice_set_state: truncated blob"); return LPC_ERR_INVALID; }
    Entry en(h);
    lpc_status st = ensure_history(h, hd.steps + 1);
    if (st != LPC_OK) return st;
    const char* p = (const char*)buf + sizeof hd;
    const size_t N = (size_t)h->N;
    void* tmp = dalloc(h, N * 8);
    if (!tmp) { set_error("lattice_set_state: temporary allocation failed"); return LPC_ERR_OOM; }
    LatticeView v = make_view(h, h->cur);
    cudaError_t e = cudaMemcpyAsync(tmp, p, N * 4, cudaMemcpyHostToDevice, h->wstream);
    if (e == cudaSuccess) e = launch_pad(tmp, 4, v, h->rho[h->cur], h->wstream);
    p += N * 4;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, p, N * 8, cudaMemcpyHostToDevice, h->wstream);
    if (e == cudaSuccess) e = launch_pad(tmp, 8, v, h->m[h->cur], h->wstream);
    p += N * 8;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        if (!(h->p.msd_axes >> a & 1)) continue;
        e = cudaStreamSynchronize(h->wstream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, p, N * 4, cudaMemcpyHostToDevice, h->wstream);
        if (e == cudaSuccess) e = launch_pad(tmp, 4, v, h->mu[h->cur][a], h->wstream);
        p += N * 4;
    }
    const size_t S = (size_t)hd.steps;
    for (int set = 0; set <= h->nreg && e == cudaSuccess; ++set) {
        e = cudaMemcpyAsync(h->histM + set * h->cap, p, (S + 1) * 16, cudaMemcpyHostToDevice, h->wstream);
        p += (S + 1) * 16;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->histP + set * h->cap, p, (S + 1) * 8, cudaMemcpyHostToDevice, h->wstream);
        p += (S + 1) * 8;
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            if (!(h->p.msd_axes >> a & 1)) continue;
            if (S > 0)
                e = cudaMemcpyAsync(h->histD + (set * 3 + a) * h->cap, p, S * 8, cudaMemcpyHostToDevice, h->wstream);
            p += S * 8;
        }
    }
    const long long dstep = hd.steps;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dstep, &dstep, 8, cudaMemcpyHostToDevice, h->wstream);
    // the region pass takes dMSD_r of the current state ahead of its step (the
    // blob holds steps entries): recompute entry `steps` of dMSD_r only
    if (e == cudaSuccess)
        e = launch_region_sums(updated_view(h, h->cur), h->p.weight_dtype, h->rpart, h->counter + 12, true, h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    dfree(h, tmp, N * 8);
    if (e != cudaSuccess) return cuda_fail(e, "lattice_set_state");
    h->steps = hd.steps;
    return LPC_OK;
}

lpc_status lattice_equilibrate(lpc_lattice* h, double threshold, int64_t max_iter, int32_t check_every,
                               int64_t* iters, double* max_diff) {
    Range nvtx("lattice_equilibrate");
    if (!h) { set_error("lattice_equilibrate: NULL handle"); return LPC_ERR_INVALID; }
    if (!(threshold >= 0.0) || max_iter < 0 || check_every < 1) { set_error("lattice_equilibrate: bad arguments"); return LPC_ERR_INVALID; }
    if (h->steps != 0) { set_error("lattice_equilibrate: only before the propagation phase (steps_done must be 0)"); return LPC_ERR_STATE; }
    if (h->slab) { set_error("lattice_equilibrate: the convergence check of a slab needs the whole lattice"); return LPC_ERR_STATE; }
    Entry en(h);
    lpc_status st = ensure_history(h, (long long)check_every + 2);
    if (st != LPC_OK) return st;
    long long done = 0;
    double diff = INFINITY;
    cudaError_t e = cudaSuccess;
    // with the one-step TMA schedule, rho alone is propagated (m and mu are
    // rebuilt from rho below); otherwise full steps of the one-step kernel
    const bool rho_only = h->kernel == LPC_KERNEL_TB && h->kdepth == 1;
    if (rho_only) {
        st = ensure_maps(h);
        if (st != LPC_OK) return st;
    }
    while (done < max_iter) {
        const long long chunk = (max_iter - done) < check_every ? (max_iter - done) : check_every;
        const long long zero = 0;
        e = cudaMemcpyAsync(h->dstep, &zero, 8, cudaMemcpyHostToDevice, h->wstream);
        if (e != cudaSuccess) break;
        for (long long i = 0; i < chunk && st == LPC_OK && e == cudaSuccess; ++i) {
            if (rho_only) {
                e = launch_tma1(make_view(h, h->cur), h->p.weight_dtype, *h->maps[h->cur], h->counter + 1,
                                h->wstream, true);
                h->cur ^= 1;
            } else {
                st = launch_one(h, h->wstream);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "equilibration step launch");
        if (st != LPC_OK) return st;
        done += chunk;
        e = launch_maxdiff(h->rho[h->cur], h->rho[h->cur ^ 1], make_view(h, h->cur), h->scratch, h->wstream);
        unsigned int bits = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, h->scratch, 4, cudaMemcpyDeviceToHost, h->wstream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
        if (e != cudaSuccess) break;
        float f;
        memcpy(&f, &bits, 4);
        diff = f;
        if (diff < threshold) break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "lattice_equilibrate");
    // restart the propagation phase from the equilibrated populations:
    // m = rho, mu = 0 in both buffers, step counter -1, then the n = 0 sums
    const long long minus_one = -1;
    e = cudaMemcpyAsync(h->dstep, &minus_one, 8, cudaMemcpyHostToDevice, h->wstream);
    if (e == cudaSuccess) e = launch_restart(make_view(h, h->cur), h->wstream);
    if (e == cudaSuccess) e = launch_reservoir_ghosts(make_view(h, h->cur), h->rf, h->wstream);
    if (e == cudaSuccess) e = launch_sum_state(updated_view(h, h->cur), h->wstream);
    if (e == cudaSuccess)
        e = launch_region_sums(updated_view(h, h->cur), h->p.weight_dtype, h->rpart, h->counter + 12, false, h->wstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->wstream);
    if (e != cudaSuccess) return cuda_fail(e, "lattice_equilibrate");
    {
        const lpc_status ds = check_device_error(h);
        if (ds != LPC_OK) return ds;
    }
    if (iters) *iters = done;
    if (max_diff) *max_diff = diff;
    return LPC_OK;
}

}  // extern "C"
