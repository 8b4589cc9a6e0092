/*
 * lpc3d.h -- C ABI of the B300 (sm_103a) lattice-propagation library.
 *
 * The library advances the lattice-gas / moment-propagation model of LPC3D
 * (arXiv 2603.22553) on one GPU.  Per time step, for every site y of an
 * nx x ny x nz simple cubic lattice (Sec. 2.1, Fig. 1):
 *
 *   rho'(y) = s(y) rho(y) + sum_k w_k(y - e_k) rho(y - e_k)
 *   m'(y)   = R(y) [ s(y) m(y) + sum_k w_k(y - e_k) m(y - e_k) ]
 *   mu_a'(y)= s(y) mu_a(y) + sum_k w_k(y - e_k) [ mu_a(y - e_k) + d_ka rho(y - e_k) ]
 *
 * with the six neighbour offsets e_k (k = +x, -x, +y, -y, +z, -z), the hop
 * weight w_k(x) = (alpha/6) * P(x -> x + e_k) from the Metropolis rule of
 * Eq. 1 (zero towards a solid site or across a wall), the stay weight
 * s(x) = 1 - sum_k w_k(x) (Sec. 2.1: a rejected move leaves the particle in
 * place; alpha is the jump factor of Eq. 7), the rotation R(y) =
 * exp(i omega(y) dt) of the destination site (Eq. 8, 11, 13), and the first
 * displacement moment mu_a used for the mean-square displacement (moment
 * propagation, Sec. 2.2; d_ka = +1 / -1 for a hop along +a / -a).
 *
 * Every step also reduces, in FP64 from FP32 partials,
 *   M(n) = sum_x m(x, n)                      (the FID, Eq. 12)
 *   P(n) = sum_x rho(x, n)                    (population)
 *   dMSD_a(n) = sum_x [2 (w_+a - w_-a) mu_a + (w_+a + w_-a) rho](x, n)
 * and MSD_a(n) = sum_{j<n} dMSD_a(j) / P(0) (Eq. 5 summed over steps).
 *
 * Conventions
 *  - Host arrays are C order [z][y][x] with x fastest (N = nx*ny*nz values).
 *  - Input arrays are copied during lattice_create; the caller keeps them.
 *  - Output buffers belong to the caller.  Query calls synchronise the
 *    lattice's stream before returning.
 *  - Every call returns an lpc_status and never aborts the process; on
 *    failure lpc_last_error() gives a message (thread-local).
 *  - lattice_step_n and lattice_step_many are asynchronous on the lattice's
 *    stream.
 */
#ifndef LPC3D_H
#define LPC3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpc_lattice lpc_lattice;   /* opaque; created and destroyed by the caller */

typedef enum {
    LPC_OK = 0,
    LPC_ERR_INVALID = 1,   /* bad argument or misuse; nothing was changed */
    LPC_ERR_OOM = 2,       /* the allocator returned NULL */
    LPC_ERR_CUDA = 3,      /* a CUDA call failed; the message names it */
    LPC_ERR_TIMEOUT = 4,   /* a bounded device wait ran out */
    LPC_ERR_STATE = 5      /* the handle is in a state that forbids the call */
} lpc_status;

enum { LPC_WEIGHTS_F32 = 0, LPC_WEIGHTS_BF16 = 1 };
enum { LPC_INIT_UNIFORM = 0, LPC_INIT_BOLTZMANN = 1 };
enum { LPC_KERNEL_AUTO = 0, LPC_KERNEL_STEP1 = 1, LPC_KERNEL_TB = 2 };
enum { LPC_STATIC_AUTO = 0, LPC_STATIC_GATHER = 1, LPC_STATIC_LINK = 2 };

/*
 * Device memory hooks.  alloc returns device memory of at least `bytes`
 * bytes, aligned to 256 bytes, usable on `stream` (a cudaStream_t), or NULL.
 * free releases it.  With a NULL lpc_allocator the library uses
 * cudaMallocAsync / cudaFreeAsync on the lattice's stream.
 */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* p, void* stream, void* ctx);
    void* ctx;
} lpc_allocator;

/*
 * Lattice parameters (Sec. 3.2 item 1: dimensions, time step, boundary
 * conditions).
 *   nx, ny, nz    lattice edge lengths, each >= 1; nx*ny*nz <= 2^31 - 1.
 *   periodic[a]   1 = periodic along axis a (ghost-layer semantics),
 *                 0 = wall: a move out of the domain is rejected.
 *   alpha         jump probability factor of Eq. 7, 0 < alpha <= 1.
 *   dt            time step in seconds; R = exp(i omega dt).
 *   kT            thermal energy in the units of F (> 0).
 *   weight_dtype  LPC_WEIGHTS_F32 or LPC_WEIGHTS_BF16 storage of w_k.
 *   msd_axes      bit mask of the axes whose first moment is propagated
 *                 (x = 1, y = 2, z = 4); 0 = none.
 *   init          initial population when rho0 is NULL: LPC_INIT_UNIFORM
 *                 (1 on pore sites) or LPC_INIT_BOLTZMANN (Eq. 2 with
 *                 mean 1 over pore sites).
 *   ghost         ghost-layer width in x and y: 0 = automatic (2) or an
 *                 even width 2..8 (even, so that the
 *                 two-site vector loads of the step kernels stay aligned); the
 *                 temporally blocked kernel needs ghost >= its block depth.
 */
typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
    double alpha;
    double dt;
    double kT;
    int32_t weight_dtype;
    int32_t msd_axes;
    int32_t init;
    int32_t ghost;
} lpc_params;

/* Static facts about a lattice (for sizing, admission and reporting). */
typedef struct {
    int64_t n_sites;          /* nx*ny*nz */
    int64_t n_padded;         /* sites of the ghost-padded device arrays */
    int32_t ghost;            /* ghost width in x and y */
    int32_t pitch_x;          /* padded x extent (elements) */
    int32_t pitch_y;          /* padded y extent */
    int32_t kernel;           /* LPC_KERNEL_* chosen for lattice_step_n */
    int32_t block_steps;      /* time steps per launch of that kernel */
    int32_t static_form;      /* static data of the TMA one-step kernel: 0 not made yet,
                                 1 gather form (in-weights, stay weight, R), 2 link form
                                 (one signed weight per link and axis, R) */
    int64_t device_bytes;     /* device memory held by the lattice */
    int64_t bytes_per_site_update; /* algorithmic HBM bytes of one site update (state
                                      read + write, hop weights, R, moments, region label) */
    int32_t tile_rows;        /* TMA-fed one-step kernel: rows of a 64-site-wide tile */
    int32_t items_per_cta;    /* TMA-fed one-step kernel: work items per CTA (sets the z chunk) */
} lpc_info;

/*
 * Create a lattice (Sec. 3.2 items 1-2: fields are created from the site
 * free energies F, frequencies omega and the solid mask; hop weights are
 * packed once from Eq. 1 and Eq. 7, rotation factors R are computed in
 * FP64 and rounded to FP32).
 *   F       [N] double, free energy of every site (kT units when kT = 1);
 *           must be finite on pore sites, ignored on solid sites.
 *   omega   [N] double, angular frequency in rad/s (finite).
 *   solid   [N] uint8, nonzero = solid (inaccessible) site.
 *   rho0    [N] double initial population or NULL (see params.init); solid
 *           sites are forced to 0.  m(x, 0) = rho(x, 0), mu(x, 0) = 0.
 *   a       allocator or NULL.   stream: cudaStream_t or NULL (default).
 *   out     receives the handle (NULL on failure).
 * Records M(0) and P(0).  Errors: LPC_ERR_INVALID (bad shape, alpha outside
 * (0, 1], non-finite inputs on pore sites, NULL arrays), LPC_ERR_OOM,
 * LPC_ERR_CUDA.
 */
lpc_status lattice_create(const lpc_params* p, const double* F, const double* omega,
                          const uint8_t* solid, const double* rho0, const lpc_allocator* a,
                          void* stream, lpc_lattice** out);

/*
 * lattice_create with a jump factor per link (position-dependent
 * diffusivity, Sec. 2.1 after Eq. 7: alpha_ij = alpha_ji, the same factor for
 * both directions of a link, so that detailed balance and the Boltzmann
 * equilibrium of Eq. 2 are kept).
 *   alpha_links  [3][N] double, host, C order per axis: alpha_links[a*N + i]
 *                is the factor of the link between site i and its +a
 *                neighbour (a = 0: x, 1: y, 2: z; the neighbour wraps on a
 *                periodic axis, the value is unused across a wall); each in
 *                [0, 1] (0 closes the link).  NULL: params.alpha on every link.
 * The hop weight is w_k(x) = alpha_link / 6 * min(1, exp(-dF/kT)).  Other
 * arguments, ownership and errors as lattice_create; LPC_ERR_INVALID for a
 * factor outside [0, 1].  The copy of alpha_links (24 bytes per site) is
 * transient, like those of F and omega.
 */
lpc_status lattice_create_links(const lpc_params* p, const double* F, const double* omega,
                                const uint8_t* solid, const double* rho0, const double* alpha_links,
                                const lpc_allocator* a, void* stream, lpc_lattice** out);

/*
 * Reservoir face (Sec. 3.2 item 1: on a non-periodic boundary the field
 * values in the ghost layer are held fixed).  A reservoir is the layer of
 * ghost sites just outside one face of the domain, each holding the fixed
 * population rho, magnetisation (m_re, m_im) and first moment 0 at every
 * step, with free energy F.  A boundary pore site exchanges population with
 * its reservoir site by the Metropolis rule of Eq. 1: out-weight
 * alpha/6 * min(1, exp(-(F - F_site)/kT)), in-weight
 * alpha/6 * min(1, exp(-(F_site - F)/kT)) times the reservoir's state
 * (alpha is params.alpha on reservoir links).  With every reservoir at the
 * same (F, rho) the state rho(x) = rho exp(-(F(x) - F)/kT) is stationary.
 */
typedef struct {
    int32_t enabled;      /* 1 = reservoir on this face, 0 = wall */
    int32_t reserved;     /* must be 0 */
    double F;             /* free energy of the reservoir sites (finite) */
    double rho;           /* fixed population of a reservoir site (finite) */
    double m_re, m_im;    /* fixed magnetisation of a reservoir site (finite) */
} lpc_reservoir;

#define LPC_MAX_REGIONS 4

/*
 * Options of lattice_create_ex (zero-initialise the struct for none).
 *   alpha_links  [3][N] per-link jump factors or NULL (as lattice_create_links).
 *   reservoir[f] face f = 2 a + side of axis a (0 = x, 1 = y, 2 = z; side 0
 *                is the face below coordinate 0, side 1 the face above
 *                n_a - 1).  A reservoir needs periodic[a] = 0.  x and y
 *                reservoirs live in the ghost bands of the padded planes; a
 *                z reservoir is a halo plane of reservoir sites below or above
 *                the lattice (the device arrays then hold nz + 2 planes, and
 *                the other z face, without a reservoir, gets an all-solid
 *                halo plane: a wall); queries still return the nz planes.
 *   region       [N] uint8 site labels, each < n_regions, or NULL: region-
 *                resolved FID, population and MSD sums (the spectra and
 *                diffusion of separate parts of a system, e.g. bulk and
 *                electrodes, Sec. 4).  Copied at create (1 byte per site is
 *                kept on the device).
 *   n_regions    1..LPC_MAX_REGIONS with region, 0 without.
 */
typedef struct {
    const double* alpha_links;
    lpc_reservoir reservoir[6];
    const uint8_t* region;
    int32_t n_regions;
    int32_t reserved;     /* must be 0 */
} lpc_options;

/*
 * lattice_create with options (o may be NULL: then it is lattice_create).
 * Lattices with a reservoir face or with regions run the one-step kernels
 * (lattice_set_schedule rejects TB with block_steps > 1 for them).  A z
 * reservoir copies the fields into nz + 2 planes on the host during create
 * (transient).  Other arguments, ownership and errors as lattice_create;
 * LPC_ERR_INVALID also for a reservoir on a periodic axis, non-finite
 * reservoir values, region labels >= n_regions, or n_regions outside 1..4
 * with region (0 without).
 */
lpc_status lattice_create_ex(const lpc_params* p, const lpc_options* o, const double* F,
                             const double* omega, const uint8_t* solid, const double* rho0,
                             const lpc_allocator* a, void* stream, lpc_lattice** out);

/*
 * Slab of a lattice decomposed along z (the slowest axis), for running one
 * lattice on several GPUs (or as several handles on one): the paper runs
 * large systems as domain-decomposed processes with ghost layers exchanged
 * between neighbours (Sec. 3.2-3.3).  A slab holds its own nz planes plus
 * one halo plane on each side: the plane just below its first plane and the
 * plane just above its last, copies of the neighbouring slabs' boundary
 * planes.  Its steps read the halos and never write them; they update and
 * sum over the own planes only, so the slabs' M, P and dMSD histories add up
 * to the whole lattice's.
 *   p        the slab's parameters: nx, ny as the lattice, nz = the slab's
 *            own planes; periodic[2] is ignored (the halo planes bound the
 *            slab), periodic[0..1] as the lattice.
 *   halo     halo planes per side; must be 1 (one step between exchanges).
 *   F, omega, solid, rho0   [nz + 2][ny][nx]: plane 0 is the lower halo
 *            (the lattice's plane below the slab; the last plane when z is
 *            periodic and this is the first slab), planes 1..nz the slab's
 *            own, plane nz + 1 the upper halo.  At a z wall of the lattice
 *            the halo plane there is all solid (solid = 1), so no hop crosses
 *            it and it never needs an exchange.  The hop weights between a
 *            halo and the own planes are packed from these fields, exactly as
 *            in the whole lattice.
 *   o        options as lattice_create_ex; region labels are not accepted.
 * A slab needs rho0 with LPC_INIT_BOLTZMANN (the normalisation of Eq. 2 is
 * over the whole lattice).  Steps: lattice_step_n advances the own planes;
 * between two steps the caller refreshes the halos from the neighbours
 * (lattice_slab_planes gives the device addresses; a step's results are in
 * place once lattice_step_n returns on the caller's stream), so a slab is
 * advanced one step at a time.  Schedules: the one-step kernels (TB with
 * block_steps > 1 is rejected); lattice_equilibrate is rejected
 * (LPC_ERR_STATE: its convergence check needs every slab).  Queries
 * (densities, weights, rotation, solid mask, lattice_info.n_sites) cover the
 * own planes; checkpoints (lattice_get_state / lattice_set_state) hold every
 * plane, halos included.  lattice_footprint of the parameters with nz + 2
 * planes gives the slab's device bytes.  Errors as lattice_create_ex, and
 * LPC_ERR_INVALID for halo != 1, region labels, or LPC_INIT_BOLTZMANN without
 * rho0.
 */
lpc_status lattice_create_slab(const lpc_params* p, int32_t halo, const lpc_options* o, const double* F,
                               const double* omega, const uint8_t* solid, const double* rho0,
                               const lpc_allocator* a, void* stream, lpc_lattice** out);

/* Planes of a slab, for the halo exchange. */
enum { LPC_PLANE_FIRST = 0, LPC_PLANE_LAST = 1, LPC_PLANE_HALO_BELOW = 2, LPC_PLANE_HALO_ABOVE = 3 };

/*
 * Device addresses of one plane of the current state of a slab.  plane[q]
 * and bytes[q] for q = rho (FP32), m (FP32 (re, im) pairs), mu_x, mu_y,
 * mu_z (FP32; NULL and 0 when the moment is not enabled).  A plane is the
 * whole ghost-padded plane (pitch_y rows of pitch_x sites, lattice_info), so
 * a copy of it carries the x / y ghost images too.  The exchange after a step
 * copies every slab's LPC_PLANE_FIRST plane into the LPC_PLANE_HALO_ABOVE
 * plane of the slab below it and its LPC_PLANE_LAST plane into the
 * LPC_PLANE_HALO_BELOW plane of the slab above it (byte copies; the slabs
 * share nx, ny, the ghost width and the moments).  The addresses change with
 * every step (the state is double-buffered): ask again after each step.
 * Copies issued on the lattice's caller stream after lattice_step_n are
 * ordered after that step, and the next step after them.  Errors:
 * LPC_ERR_INVALID (NULL arguments, a lattice that is not a slab, which
 * outside 0..3).
 */
typedef struct {
    void* plane[5];
    int64_t bytes[5];
} lpc_plane_set;
lpc_status lattice_slab_planes(lpc_lattice* h, int32_t which, lpc_plane_set* out);

/*
 * Device bytes lattice_create would hold for these parameters, plus the
 * history of `steps` steps and the transient input copies of create (used to
 * admit requests by HBM footprint).  No device work.  LPC_ERR_INVALID on bad
 * parameters.  Options of lattice_create_ex add to it: per-link factors
 * 24 bytes per site during create; region labels 1 byte per site, one more
 * history set (48 bytes per step) per region and 4x the per-item partial
 * sums (about 7 MB).
 */
lpc_status lattice_footprint(const lpc_params* p, int64_t steps, int64_t* bytes);

/* Release every device buffer of the lattice.  NULL-safe. */
lpc_status lattice_destroy(lpc_lattice* h);

/*
 * Advance n >= 0 time steps (Sec. 3.2 item 4, the propagation phase),
 * recording M, P and dMSD for every step.  Asynchronous on the lattice's
 * stream; may grow the device history buffers (via the allocator) before
 * launching.  Errors: LPC_ERR_INVALID (NULL handle, n < 0), LPC_ERR_OOM,
 * LPC_ERR_CUDA.
 */
lpc_status lattice_step_n(lpc_lattice* h, int64_t n);

/*
 * Advance several lattices (all on one device); lattice i by n[i] steps.
 * Each step is one batched launch over the work items of up to 48 lattices
 * (grouped by weight type and MSD mask), so many small lattices fill the
 * GPU together.  States are bit-identical to lattice_step_n; the per-step
 * sums agree with it to FP32 rounding and are bit-identical whether a
 * lattice is advanced alone or with any other lattices.  The launches wait
 * for the work queued on every lattice's stream; later calls on these
 * lattices (queries included) are ordered after them.  Work the caller
 * queues on its own stream is ordered after them only through
 * lattice_sync or a query.  Errors: LPC_ERR_INVALID (NULL or repeated
 * handle, negative n, lattices on different devices), LPC_ERR_OOM,
 * LPC_ERR_CUDA.
 */
lpc_status lattice_step_many(lpc_lattice* const* hs, const int64_t* n, int32_t count);

/* Choose the step kernel: LPC_KERNEL_AUTO (the default: the TMA-fed
 * one-step kernel for lattices of at least 2^20 sites with nx >= 64 and
 * ny >= 16, else the register-pipelined one, which is faster on smaller
 * lattices), STEP1, or TB with block depth
 * k (1..min(4, ghost); k = 1 is the TMA-fed one-step kernel).
 * LPC_ERR_INVALID if the combination is impossible. */
lpc_status lattice_set_schedule(lpc_lattice* h, int32_t kernel, int32_t block_steps);

/*
 * Form of the static data (hop weights and R) read by the TMA-fed one-step
 * kernel (the automatic schedule of large lattices, or lattice_set_schedule
 * (LPC_KERNEL_TB, 1)).  Both forms hold the weights packed from Eq. 1 and
 * Eq. 7 exactly, so states are bit-identical in either; they differ in the
 * bytes a site update reads:
 *   LPC_STATIC_GATHER  per site the six in-weights w_k(y - e_k), the stay
 *                      weight and R (gather form);
 *   LPC_STATIC_LINK    one signed weight per link and axis, and R (link
 *                      form): one hop of every open link is a downhill or
 *                      level Metropolis move of weight alpha/6 (Eq. 1), so
 *                      one number gives both; the kernel rebuilds in-, out-
 *                      and stay weights from it.  Needs one jump factor (no
 *                      per-link factors); reservoir links follow the same
 *                      rule, and region labels are read beside the links;
 *   LPC_STATIC_AUTO    the default: the link form for FP32 lattices of at
 *                      least 3 * 2^24 sites that allow it, else the gather
 *                      form.
 * Static data made earlier in another form is released.  When the lattice's
 * schedule is the TMA-fed one-step kernel the chosen form is made during this
 * call (synchronously), else on that kernel's first launch.  Errors:
 * LPC_ERR_INVALID (NULL handle, unknown form, LPC_STATIC_LINK for a lattice
 * with per-link jump factors), LPC_ERR_OOM, LPC_ERR_CUDA.
 */
lpc_status lattice_set_static_form(lpc_lattice* h, int32_t form);

/*
 * Tiling of the TMA-fed one-step kernel: tile_rows (8, 12 or 16: a tile is
 * 64 x tile_rows sites, one consumer warp per row) and items_per_cta (work
 * items per CTA of the persistent grid, which sets the z-chunk length of an
 * item: chunks of at least 8 planes).  0 keeps the heuristic (the tallest
 * tile whose shared-memory rings keep 3 planes in flight; 40 items per CTA).
 * A tile height whose rings do not fit falls back to the heuristic
 * (lattice_info reports the one used).  States do not depend on the tiling;
 * sums agree to FP32 summation order.  Errors: LPC_ERR_INVALID.
 */
lpc_status lattice_set_tiling(lpc_lattice* h, int32_t tile_rows, int32_t items_per_cta);

/*
 * Autotune the step schedule of this lattice: times `trial_launches`
 * launches of every candidate with CUDA events (the register-pipelined
 * one-step kernel; the TMA-fed one-step kernel at tile rows 16, 12, 8 and
 * 20, 40, 80 work items per CTA; TB with depth 2..min(4, ghost)), keeps the
 * fastest and restores the lattice's state, step counter and history
 * afterwards (results are as if no trial had run).  kernel / block_steps /
 * rate (nullable) receive the choice and its site updates per second; the
 * tiling is in lattice_info.  Errors: LPC_ERR_INVALID, LPC_ERR_OOM (state
 * snapshot), LPC_ERR_CUDA.
 */
lpc_status lattice_autotune(lpc_lattice* h, int32_t trial_launches, int32_t* kernel,
                            int32_t* block_steps, double* rate);

/* Wait for all queued work of the lattice. */
lpc_status lattice_sync(lpc_lattice* h);

/* Number of time steps completed (queued steps count once queued). */
lpc_status lattice_steps_done(lpc_lattice* h, int64_t* n);

/* Static facts about the lattice. */
lpc_status lattice_info(lpc_lattice* h, lpc_info* out);

/*
 * FID samples M(n) for n = first .. first+count-1 (Eq. 12; G(n) = M(n)/P(0)
 * is the normalised FID of Eq. 8 / Eq. 11).  out: 2*count doubles,
 * (re, im) pairs, host memory.  LPC_ERR_INVALID if the range exceeds the
 * steps done (0 .. steps_done inclusive).
 */
lpc_status lattice_fid(lpc_lattice* h, int64_t first, int64_t count, double* out);

/* Population P(n) = sum_x rho(x, n), same range rules as lattice_fid. */
lpc_status lattice_population(lpc_lattice* h, int64_t first, int64_t count, double* out);

/*
 * Region-resolved sums of a lattice created with region labels: the FID
 * M_r(n) = sum of m(x, n) over the sites x labelled r (out: 2*count doubles,
 * re/im), the population P_r(n), and MSD_r,a(n) = sum_{j<n} dMSD_r,a(j) / P(0)
 * with dMSD_r,a(j) the MSD increment of Eq. 5 summed over the sites labelled r
 * at step j (the part of MSD_a(n) accrued while the particles were in region
 * r; the regions add up to lattice_msd).  Sums over r equal lattice_fid,
 * lattice_population and lattice_msd up to FP64 rounding.  Range rules as
 * lattice_fid; LPC_ERR_INVALID for a region >= n_regions or a lattice
 * without regions.
 */
lpc_status lattice_fid_region(lpc_lattice* h, int32_t region, int64_t first, int64_t count, double* out);
lpc_status lattice_population_region(lpc_lattice* h, int32_t region, int64_t first, int64_t count,
                                     double* out);
lpc_status lattice_msd_region(lpc_lattice* h, int32_t region, int32_t axis, int64_t first, int64_t count,
                              double* out);

/*
 * Mean-square displacement along `axis` (0 = x, 1 = y, 2 = z):
 * MSD_a(n) = sum_{j<n} dMSD_a(j) / P(0) for n = first .. first+count-1,
 * from moment propagation (Sec. 2.2, Eq. 5); D = MSD / (2 n dt) per axis.
 * LPC_ERR_INVALID if the axis is not in msd_axes or the range is invalid.
 */
lpc_status lattice_msd(lpc_lattice* h, int32_t axis, int64_t first, int64_t count, double* out);

/*
 * The per-step MSD increments dMSD_a(n) = sum_x [2 (w_+a - w_-a) mu_a +
 * (w_+a + w_-a) rho](x, n) of Eq. 5 (summed over the lattice's sites, or a
 * slab's own planes) for n = first .. first+count-1 (0 .. steps_done - 1):
 * the values lattice_msd accumulates, unnormalised, so that the increments
 * of several slabs can be added before dividing by the whole lattice's P(0).
 * LPC_ERR_INVALID if the axis is not in msd_axes or the range is invalid.
 */
lpc_status lattice_dmsd(lpc_lattice* h, int32_t axis, int64_t first, int64_t count, double* out);

/*
 * Current site populations rho(x, n) (the densities of Sec. 3.2 item 5),
 * N floats, C order.  out_is_device = 1: `out` is device memory (copied on
 * the lattice's stream), 0: host memory.
 */
lpc_status lattice_density(lpc_lattice* h, float* out, int32_t out_is_device);

/* Current magnetisation m(x, n): N (re, im) float pairs. */
lpc_status lattice_magnetization(lpc_lattice* h, float* out, int32_t out_is_device);

/* Current first moment mu_axis(x, n): N floats; the axis must be enabled. */
lpc_status lattice_moment(lpc_lattice* h, int32_t axis, float* out, int32_t out_is_device);

/*
 * Packed hop weights as stored, widened to float: out[k*N + i] = w_k(site i)
 * for k = +x, -x, +y, -y, +z, -z (6*N floats, host).  Solid sites and moves
 * into solids or across walls are exactly 0 (the geometry of Fig. 1).
 */
lpc_status lattice_weights(lpc_lattice* h, float* out);

/* Rotation factors R(x) = exp(i omega dt) as stored: N (re, im) float pairs. */
lpc_status lattice_rotation(lpc_lattice* h, float* out);

/* Solid mask as stored on the device: N bytes (0 pore, 1 solid). */
lpc_status lattice_solid(lpc_lattice* h, uint8_t* out);

/*
 * Checkpoint / resume.  The state blob holds rho, m, mu (FP32, interior
 * sites), the step counter and the FP64 histories (totals and regions);
 * lattice_state_size gives its size.  lattice_set_state requires a lattice created with the same
 * parameters.  Resuming and running m more steps gives the same results,
 * bit for bit, as running them without the checkpoint.
 */
lpc_status lattice_state_size(lpc_lattice* h, size_t* bytes);
lpc_status lattice_get_state(lpc_lattice* h, void* buf, size_t bytes);
lpc_status lattice_set_state(lpc_lattice* h, const void* buf, size_t bytes);

/*
 * Equilibration phase (Sec. 3.2 item 3): advance the population only
 * (m and mu are reset to m = rho, mu = 0 afterwards and the history is
 * restarted at n = 0) until max_x |rho(x, t+1) - rho(x, t)| < threshold,
 * checked every check_every steps, or until max_iter steps.  iters and
 * max_diff (nullable) receive the steps taken and the last difference.
 */
lpc_status lattice_equilibrate(lpc_lattice* h, double threshold, int64_t max_iter,
                               int32_t check_every, int64_t* iters, double* max_diff);

/*
 * One time step that allocates no device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory where they advance the lattice (host codes whose device
 * memory is reserved once through their own pool, plain C hosts without
 * allocator hooks).  The caller owns every buffer; all are device memory in
 * plain C order [z][y][x] (no ghost padding), N = nx*ny*nz:
 *   w        [6][N] float: packed out-weights w_k (k = +x, -x, +y, -y, +z,
 *            -z), zero across walls, as lattice_weights returns them.
 *   R        [N] (re, im) float pairs: rotation factors (lattice_rotation).
 *   rho_in / m_in    state at step n (m as (re, im) float pairs).
 *   rho_out / m_out  state at step n+1; must not alias the inputs.
 *   sums     3 doubles written with M(n+1) re, M(n+1) im, P(n+1).
 *   periodic[3]      1 = periodic, 0 = wall, per axis; must be the flags the
 *            weights were packed with (weights packed for a periodic axis but
 *            stepped as a wall lose the population that hops out of the
 *            domain, and nothing detects it).
 *   stream   cudaStream_t (NULL = default stream); the call is asynchronous.
 * Alignment: R, m_in, m_out and sums 8-byte aligned; w, rho_in and rho_out
 * 4-byte aligned (LPC_ERR_INVALID otherwise, before any launch).
 * The state equals lattice_step_n by one step bit for bit (the same per-site
 * arithmetic); M and P are FP64 sums of FP32 per-row partials in plane order,
 * equal to lattice_fid / lattice_population to FP32 summation order.
 * One 256-thread block per z plane: throughput scales with nz (an nz = 1
 * lattice runs on one SM), so the call suits callers bound by their
 * allocation rules rather than by speed; lattice_step_n is the fast path.
 * Scratch: per-plane partial sums and a completion counter in a fixed
 * device array of this library (about 98 KB, held by every GPU that loads
 * the library until exit); hence nz <= 4096, and larger nz is rejected with
 * LPC_ERR_INVALID.  Every call looks up that array's address
 * (cudaGetSymbolAddress, a host-side lookup); the first call on a device also
 * loads the library's device code there, so make a first call before any
 * stream capture.  Calls share the array: calls that overlap on the GPU race
 * and give wrong sums, so order them.  No MSD moments.  Errors:
 * LPC_ERR_INVALID (sizes, NULL, aliased or misaligned buffers), LPC_ERR_CUDA.
 */
lpc_status lpc_step_noalloc(int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                            const float* w, const float* R, const float* rho_in, const float* m_in,
                            float* rho_out, float* m_out, double* sums, void* stream);

/*
 * Failure-detection self-test (the paper has no counterpart).  Every
 * spin-wait of the step kernels is bounded by an SM clock budget: a wait that
 * runs out writes LPC_ERR_TIMEOUT to the lattice's status word and the kernel
 * returns, so the context stays usable and the next query reports the error.
 * This call runs one such bounded wait in a one-thread kernel on `stream`
 * (cudaStream_t, NULL = default stream) and waits for it:
 *   mode 0   a shared-memory mbarrier that never completes (no arrival);
 *   mode 1   a device flag that nothing sets;
 *   mode 2   an mbarrier that completes before the wait (control).
 * budget_cycles (1 .. 4e9; 4e9 is the step kernels' bound, about 2 s) is
 * the SM clock cycles the wait may take.  Returns LPC_ERR_TIMEOUT when the
 * wait ran out (modes 0 and 1), LPC_OK when it ended (mode 2).  Allocates
 * and frees 8 bytes of device memory.  Errors: LPC_ERR_INVALID (mode or
 * budget out of range), LPC_ERR_CUDA.
 */
lpc_status lpc_wait_selftest(int32_t mode, int64_t budget_cycles, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* lpc_last_error(void);

/* Library version string. */
const char* lpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LPC3D_H */
