/*
 * FP64 CPU oracle for the lattice-gas / moment-propagation step of LPC3D
 * (arXiv 2603.22553).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the CPU baseline of the benchmark.  It shares no code, header or
 * constant with the CUDA library; the two meet only through seeded inputs.
 *
 * What it computes (plain definitions, no blocking or fusion):
 *
 *  Hop weights (Sec. 2.1, Fig. 1, Eq. 1; Eq. 7 for alpha):
 *    each of the z = 6 neighbours is attempted with probability 1/6; a move
 *    is accepted with the Metropolis probability of Eq. 1 (1 when the target
 *    free energy is not higher, exp(-dF/kT) otherwise) and scaled by the jump
 *    factor alpha of Eq. 7.  A move towards a solid site, or out of the
 *    domain across a non-periodic face, is rejected (weight 0); the particle
 *    stays.  w_k(x) = (alpha/6) * P(x -> x+e_k) and the stay weight is
 *    s(x) = 1 - sum_k w_k(x).
 *    Position-dependent diffusivity (Sec. 2.1, after Eq. 7): alpha may be
 *    given per link, alpha_ij = alpha_ji, the same factor for both
 *    directions of a link so that detailed balance holds; it is stored once
 *    per link as alpha_links[a][i] for the link between site i and its +a
 *    neighbour (a = x, y, z).
 *    Reservoir faces (Sec. 3.2 item 1: non-periodic boundaries with field
 *    values fixed in the ghost layer): on a non-periodic axis each of the two
 *    faces may hold a reservoir, a layer of virtual sites just outside the
 *    domain with a fixed free energy F_res, population rho_res and
 *    magnetisation m_res (first moment 0).  A boundary pore site exchanges
 *    population with it by the same Metropolis rule: out-weight
 *    (alpha/6) min(1, exp(-(F_res - F_i)/kT)), in-weight
 *    (alpha/6) min(1, exp(-(F_i - F_res)/kT)) times the reservoir's fixed
 *    state.  Reservoir links use the scalar alpha.  A face without a
 *    reservoir is a wall.
 *
 *  One step (master equation of the average densities, Sec. 2.1 / Eq. 2, and
 *  the moment-propagation recursion of Sec. 2.2-2.3, Eq. 13 in 3D with the
 *  stay term and the 1/z attempt factor):
 *    rho'(y) = s(y) rho(y) + sum_k w_k(y-e_k) rho(y-e_k)
 *    m'(y)   = R(y) [ s(y) m(y) + sum_k w_k(y-e_k) m(y-e_k) ],
 *              R(y) = exp(i omega(y) dt)   (Eq. 8, 11, 13: the phase of the
 *              destination site, applied after the hop)
 *    mu_a'(y) = s(y) mu_a(y) + sum_k w_k(y-e_k) [mu_a(y-e_k) + d_ka rho(y-e_k)]
 *              (first moment of the displacement along axis a, d_ka = +1 / -1
 *              when e_k points along +a / -a, else 0: Sec. 2.2)
 *
 *  Per-step sums (Eq. 12, Eq. 5):
 *    M(n) = sum_x m(x, n), P(n) = sum_x rho(x, n),
 *    dMSD_a(n) = sum_x [2 (w_+a - w_-a)(x) mu_a(x, n) + (w_+a + w_-a)(x) rho(x, n)]
 *    so that MSD_a(n) = sum_{j<n} dMSD_a(j) / P(0).
 *  Region-resolved sums (the spectra and diffusion of separate parts of the
 *  system, bulk and electrodes, Sec. 4): every site carries a label r, and
 *  M_r(n), P_r(n) and dMSD_a,r(n) are the same sums restricted to the sites
 *  labelled r at step n.  They add up to M, P and dMSD.
 *
 * Readings of the paper taken here: Eq. 13 as printed has no stay term and no
 * 1/z factor; the full master-equation form above conserves population as the
 * text requires.  omega is an angular frequency (rad/s); R = exp(+i omega dt).
 * Ties in Eq. 1 (E_j = E_i) accept.
 *
 * Layout: C order [z][y][x], x fastest; weights w[site*6 + k] with
 * k = 0:+x 1:-x 2:+y 3:-y 4:+z 5:-z.  Sums are taken per z-plane in a fixed
 * order and then over planes in z order, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <fenv.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_INVALID 1

/* Round a double to the nearest value with `bits` significand bits
 * (ties to even): bits = 24 is IEEE binary32, bits = 8 is bfloat16.  Only used
 * for finite values inside the normal range of the target format. */
static double round_sig(double v, int bits)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double f = frexp(v, &e);              /* v = f * 2^e, 0.5 <= |f| < 1 */
    double scaled = ldexp(f, bits);       /* |scaled| in [2^(bits-1), 2^bits) */
    double r = nearbyint(scaled);         /* default mode: nearest, ties even */
    return ldexp(r, e - bits);
}

double or_round_f32(double v) { return round_sig(v, 24); }
double or_round_bf16(double v) { return round_sig(v, 8); }

static int64_t site(int x, int y, int z, int nx, int ny) { return ((int64_t)z * ny + y) * nx + x; }

/* Neighbour of (x, y, z) along direction k, or -1 when it lies outside a
 * non-periodic face. */
static int64_t neighbour(int x, int y, int z, int k, int nx, int ny, int nz, const int* periodic)
{
    static const int off[6][3] = {{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
    int c[3] = {x + off[k][0], y + off[k][1], z + off[k][2]};
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (!periodic[a]) return -1;
            c[a] = (c[a] % n[a] + n[a]) % n[a];
        }
    }
    return site(c[0], c[1], c[2], nx, ny);
}

/*
 * Hop weights, stay weights and rotation factors.
 * mode 0: exact FP64.  mode 1: weights and R rounded to binary32.
 * mode 2: weights rounded to bfloat16, R rounded to binary32.
 * In the rounded modes s = 1 - sum of the rounded weights (in FP64).
 * alpha_links: NULL (alpha on every link) or [3][N] per-link factors in [0, 1].
 * res: NULL (no reservoir) or [6][5] per face f = 2 a + side (side 0: the face
 * below coordinate 0, side 1: the face above n_a - 1) holding
 * {enabled, F_res, rho_res, m_res re, m_res im}; a reservoir needs a
 * non-periodic axis.  wres: NULL, or [N][6] receiving the in-weight of the
 * hop along e_k into each site from a reservoir (0 where the source i - e_k
 * is not a reservoir site).
 */
int or_pack_ex(int nx, int ny, int nz, const int* periodic, double alpha, const double* alpha_links,
               double dt, double kT, int mode, const double* F, const double* omega,
               const uint8_t* solid, const double* res, double* w, double* s, double* R, double* wres)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(kT > 0.0)) return OR_INVALID;
    const int64_t N = (int64_t)nx * ny * nz;
    if (alpha_links)
        for (int64_t i = 0; i < 3 * N; ++i)
            if (!(alpha_links[i] >= 0.0 && alpha_links[i] <= 1.0)) return OR_INVALID;
    if (res)
        for (int f = 0; f < 6; ++f)
            if (res[5 * f] != 0.0 && (periodic[f >> 1] || !isfinite(res[5 * f + 1]))) return OR_INVALID;
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t i = site(x, y, z, nx, ny);
                double out = 0.0;
                for (int k = 0; k < 6; ++k) {
                    int64_t j = neighbour(x, y, z, k, nx, ny, nz, periodic);
                    double wk = 0.0;
                    if (j >= 0 && !solid[i] && !solid[j]) {
                        double dE = (F[j] - F[i]) / kT;
                        double p = (dE > 0.0) ? exp(-dE) : 1.0;   /* Eq. 1 */
                        /* the link of a +a hop starts at i, that of a -a hop at j */
                        double a_link = alpha;
                        if (alpha_links) a_link = alpha_links[(int64_t)(k >> 1) * N + ((k & 1) ? j : i)];
                        wk = a_link / 6.0 * p;
                    } else if (j < 0 && !solid[i] && res) {
                        /* a +a hop leaves through the upper face, a -a hop through the lower */
                        const double* rf = res + 5 * (2 * (k >> 1) + ((k & 1) ? 0 : 1));
                        if (rf[0] != 0.0) {
                            double dE = (rf[1] - F[i]) / kT;
                            wk = alpha / 6.0 * ((dE > 0.0) ? exp(-dE) : 1.0);
                        }
                    }
                    if (mode == 1) wk = or_round_f32(wk);
                    else if (mode == 2) wk = or_round_bf16(wk);
                    w[i * 6 + k] = wk;
                    out += wk;
                    if (wres) {
                        /* the source of a hop along e_k into i is i - e_k: below the
                         * lower face for a +a hop, above the upper face for a -a hop */
                        double wi = 0.0;
                        if (res && !solid[i] && neighbour(x, y, z, k ^ 1, nx, ny, nz, periodic) < 0) {
                            const double* rf = res + 5 * (2 * (k >> 1) + (k & 1));
                            if (rf[0] != 0.0) {
                                double dE = (F[i] - rf[1]) / kT;
                                wi = alpha / 6.0 * ((dE > 0.0) ? exp(-dE) : 1.0);
                            }
                        }
                        if (mode == 1) wi = or_round_f32(wi);
                        else if (mode == 2) wi = or_round_bf16(wi);
                        wres[i * 6 + k] = wi;
                    }
                }
                s[i] = 1.0 - out;
                double th = omega[i] * dt;
                double c = cos(th), sn = sin(th);
                if (mode != 0) { c = or_round_f32(c); sn = or_round_f32(sn); }
                R[2 * i] = c;
                R[2 * i + 1] = sn;
            }
    return OR_OK;
}

int or_pack_links(int nx, int ny, int nz, const int* periodic, double alpha, const double* alpha_links,
                  double dt, double kT, int mode, const double* F, const double* omega,
                  const uint8_t* solid, double* w, double* s, double* R)
{
    return or_pack_ex(nx, ny, nz, periodic, alpha, alpha_links, dt, kT, mode, F, omega, solid, NULL,
                      w, s, R, NULL);
}

int or_pack(int nx, int ny, int nz, const int* periodic, double alpha, double dt, double kT,
            int mode, const double* F, const double* omega, const uint8_t* solid,
            double* w, double* s, double* R)
{
    return or_pack_links(nx, ny, nz, periodic, alpha, NULL, dt, kT, mode, F, omega, solid, w, s, R);
}

/* Boltzmann densities of Eq. 2 over pore sites:
 * rho_i = mean_rho * n_pore * exp(-F_i/kT) / sum_j exp(-F_j/kT), 0 on solid. */
int or_boltzmann(int64_t N, const double* F, const uint8_t* solid, double kT, double mean_rho, double* rho)
{
    double z = 0.0;
    int64_t npore = 0;
    for (int64_t i = 0; i < N; ++i)
        if (!solid[i]) { z += exp(-F[i] / kT); ++npore; }
    if (npore == 0 || !(z > 0.0)) return OR_INVALID;
    for (int64_t i = 0; i < N; ++i)
        rho[i] = solid[i] ? 0.0 : mean_rho * (double)npore * exp(-F[i] / kT) / z;
    return OR_OK;
}

/*
 * nsteps steps from the state (rho, m, mu); the state arrays are updated in
 * place.  M has 2*(nsteps+1) entries (re, im), P has nsteps+1 entries,
 * dmsd has 3*nsteps entries laid out [axis][n] (only the axes in msd_axes,
 * bit 0 = x, 1 = y, 2 = z, are written).  mu is [3][N].
 * wres / res: the reservoir in-weights and faces of or_pack_ex (both NULL
 * when there is no reservoir); a reservoir site holds rho_res, m_res and a
 * first moment of 0 at every step.
 * region: NULL, or [N] labels < n_regions; then Mr [n_regions][nsteps+1][2],
 * Pr [n_regions][nsteps+1] and Dr [n_regions][3][nsteps] receive the
 * region-restricted sums.
 */
int or_run_ex(int nx, int ny, int nz, const int* periodic, const double* w, const double* s,
              const double* R, const double* wres, const double* res, const uint8_t* region,
              int n_regions, int msd_axes, int64_t nsteps, int nthreads,
              double* rho, double* m, double* mu, double* M, double* P, double* dmsd,
              double* Mr, double* Pr, double* Dr)
{
    if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0) return OR_INVALID;
    if ((wres == NULL) != (res == NULL)) return OR_INVALID;
    const int64_t N = (int64_t)nx * ny * nz;
    if (!region) n_regions = 0;
    if (region) {
        if (n_regions < 1 || n_regions > 256) return OR_INVALID;
        for (int64_t i = 0; i < N; ++i)
            if (region[i] >= n_regions) return OR_INVALID;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int nq = 6 * (1 + n_regions);     /* sums per plane: total, then per region */
    double* rho2 = (double*)malloc(sizeof(double) * N);
    double* m2 = (double*)malloc(sizeof(double) * 2 * N);
    double* mu2 = (double*)malloc(sizeof(double) * 3 * N);
    double* plane = (double*)malloc(sizeof(double) * nq * nz);
    double* tot = (double*)malloc(sizeof(double) * nq);
    if (!rho2 || !m2 || !mu2 || !plane || !tot) {
        free(rho2); free(m2); free(mu2); free(plane); free(tot);
        return OR_INVALID;
    }

    for (int64_t n = 0; n <= nsteps; ++n) {
        /* sums of the current state n, and the MSD increment of step n -> n+1 */
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z) {
            double* pl = plane + (int64_t)nq * z;
            for (int q = 0; q < nq; ++q) pl[q] = 0.0;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int64_t i = site(x, y, z, nx, ny);
                    double v[6] = {m[2 * i], m[2 * i + 1], rho[i], 0.0, 0.0, 0.0};
                    for (int a = 0; a < 3; ++a) {
                        if (!(msd_axes >> a & 1)) continue;
                        double wp = w[i * 6 + 2 * a], wm = w[i * 6 + 2 * a + 1];
                        v[3 + a] = 2.0 * (wp - wm) * mu[a * N + i] + (wp + wm) * rho[i];
                    }
                    for (int q = 0; q < 6; ++q) pl[q] += v[q];
                    if (region)
                        for (int q = 0; q < 6; ++q) pl[6 * (1 + region[i]) + q] += v[q];
                }
        }
        for (int q = 0; q < nq; ++q) tot[q] = 0.0;
        for (int z = 0; z < nz; ++z)
            for (int q = 0; q < nq; ++q) tot[q] += plane[(int64_t)nq * z + q];
        M[2 * n] = tot[0];
        M[2 * n + 1] = tot[1];
        P[n] = tot[2];
        for (int r = 0; r < n_regions; ++r) {
            const double* t = tot + 6 * (1 + r);
            Mr[((int64_t)r * (nsteps + 1) + n) * 2] = t[0];
            Mr[((int64_t)r * (nsteps + 1) + n) * 2 + 1] = t[1];
            Pr[(int64_t)r * (nsteps + 1) + n] = t[2];
        }
        if (n == nsteps) break;
        for (int a = 0; a < 3; ++a) {
            if (!(msd_axes >> a & 1)) continue;
            dmsd[a * nsteps + n] = tot[3 + a];
            for (int r = 0; r < n_regions; ++r)
                Dr[((int64_t)r * 3 + a) * nsteps + n] = tot[6 * (1 + r) + 3 + a];
        }

        /* the step n -> n+1 (gather form) */
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int64_t i = site(x, y, z, nx, ny);
                    double r = s[i] * rho[i];
                    double mr = s[i] * m[2 * i], mi = s[i] * m[2 * i + 1];
                    double ua[3];
                    for (int a = 0; a < 3; ++a) ua[a] = (msd_axes >> a & 1) ? s[i] * mu[a * N + i] : 0.0;
                    for (int k = 0; k < 6; ++k) {
                        /* the source of a hop along e_k into i sits at i - e_k,
                         * i.e. the neighbour of i in the opposite direction k^1 */
                        int64_t j = neighbour(x, y, z, k ^ 1, nx, ny, nz, periodic);
                        double wk, rj, mjr, mji;
                        double muj[3] = {0.0, 0.0, 0.0};
                        if (j >= 0) {
                            wk = w[j * 6 + k];
                            rj = rho[j];
                            mjr = m[2 * j];
                            mji = m[2 * j + 1];
                            for (int a = 0; a < 3; ++a)
                                if (msd_axes >> a & 1) muj[a] = mu[a * N + j];
                        } else {
                            if (!wres) continue;
                            /* reservoir site beyond the lower face (+a hop) or the upper (-a hop) */
                            const double* rf = res + 5 * (2 * (k >> 1) + (k & 1));
                            wk = wres[i * 6 + k];
                            rj = rf[2];
                            mjr = rf[3];
                            mji = rf[4];
                        }
                        r += wk * rj;
                        mr += wk * mjr;
                        mi += wk * mji;
                        int axis = k >> 1;
                        double d = (k & 1) ? -1.0 : 1.0;
                        for (int a = 0; a < 3; ++a) {
                            if (!(msd_axes >> a & 1)) continue;
                            ua[a] += wk * (muj[a] + (a == axis ? d * rj : 0.0));
                        }
                    }
                    rho2[i] = r;
                    double c = R[2 * i], sn = R[2 * i + 1];
                    m2[2 * i] = c * mr - sn * mi;
                    m2[2 * i + 1] = c * mi + sn * mr;
                    for (int a = 0; a < 3; ++a)
                        if (msd_axes >> a & 1) mu2[a * N + i] = ua[a];
                }
        memcpy(rho, rho2, sizeof(double) * N);
        memcpy(m, m2, sizeof(double) * 2 * N);
        for (int a = 0; a < 3; ++a)
            if (msd_axes >> a & 1) memcpy(mu + a * N, mu2 + a * N, sizeof(double) * N);
    }
    free(rho2); free(m2); free(mu2); free(plane); free(tot);
    return OR_OK;
}

int or_run(int nx, int ny, int nz, const int* periodic, const double* w, const double* s,
           const double* R, int msd_axes, int64_t nsteps, int nthreads,
           double* rho, double* m, double* mu, double* M, double* P, double* dmsd)
{
    return or_run_ex(nx, ny, nz, periodic, w, s, R, NULL, NULL, NULL, 0, msd_axes, nsteps, nthreads,
                     rho, m, mu, M, P, dmsd, NULL, NULL, NULL);
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
