/*
 * sp_oracle.c -- FP64 CPU oracle for the evolution of a complex scalar string
 * field on a periodic cubic lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path and imports nothing from it.
 *
 * What it computes (the plain definition the region-scheduled method must
 * reach): the whole-grid staggered leapfrog of
 *
 *     phi'' + 2 (nu / tau) phi' - Lap7 phi + a(tau)^2 lambda (|phi|^2 - eta^2) phi = 0,
 *     a(tau) = (tau / tau_ref)^nu,
 *
 * in conformal time, with the 7-point Laplacian.  The paper (Sec. 1, Sec. 2)
 * fixes the method -- spacetime cut into regions that have only initial and
 * final surfaces -- and states that the regions reproduce the evolution of
 * the whole volume; it does not fix a PDE.  The model problem and its
 * discretisation are therefore the plain textbook scheme, step n -> n+1:
 *
 *     F_n       = Lap7 phi_n / dx^2 - a_n^2 lambda (|phi_n|^2 - eta^2) phi_n
 *     pi_{n+1/2} = ((1 - d_n) pi_{n-1/2} + dt F_n) / (1 + d_n),  d_n = nu dt / tau_n
 *     phi_{n+1}  = phi_n + dt pi_{n+1/2}
 *
 * (friction term time-centred).  During an optional damping phase of
 * damp_steps levels the velocity is discarded each step (d_n = 1), tau is
 * frozen at tau0 and a = a(tau0); afterwards tau_n = tau0 + (n - damp) dt.
 *
 * Everything is FP64, whole grid, no blocking and no reordering beyond a
 * parallel loop over z-planes (each site's arithmetic is unchanged by it).
 *
 * Layout: complex fields are double[2 * nx * ny * nz], (re, im) interleaved,
 * site index x + nx * (y + ny * z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n[3];
    double dx, dt, lambda, eta, nu, tau0, tau_ref;
    int32_t damp_steps;
    int32_t reserved;
} or_params;

/* Conformal time, scale factor and friction parameter at level n. */
void or_level_coeffs(const or_params *p, int64_t level, double out[6])
{
    int damping = level < p->damp_steps;
    double tau = damping ? p->tau0 : p->tau0 + (double)(level - p->damp_steps) * p->dt;
    double ratio = tau / p->tau_ref;
    double a;
    double nu_int = floor(p->nu);
    if (p->nu == nu_int && p->nu >= 0.0 && p->nu <= 16.0) {
        a = 1.0;
        for (int i = 0; i < (int)nu_int; ++i) a *= ratio;
    } else {
        a = pow(ratio, p->nu);
    }
    double d = damping ? 1.0 : p->nu * p->dt / tau;
    out[0] = tau;
    out[1] = a;
    out[2] = d;
    out[3] = (1.0 - d) / (1.0 + d);          /* c1 */
    out[4] = p->dt / (1.0 + d);               /* c2 */
    out[5] = a * a * p->lambda;               /* m  */
}

static inline int64_t site(const int32_t n[3], int x, int y, int z)
{
    return (int64_t)x + (int64_t)n[0] * ((int64_t)y + (int64_t)n[1] * z);
}

static inline int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* One leapfrog step of the whole grid, level -> level + 1, in place. */
void or_step(const or_params *p, int64_t level, double *phi, double *pi, int nthreads)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    double co[6];
    or_level_coeffs(p, level, co);
    const double d = co[2], m = co[5];
    const double dt = p->dt, inv_dx2 = 1.0 / (p->dx * p->dx), eta2 = p->eta * p->eta;
    set_threads(nthreads);

    /* pass 1: pi_{n+1/2} from phi_n and pi_{n-1/2} (site-local write) */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t s = site(p->n, x, y, z);
                int64_t nb[6] = {
                    site(p->n, wrap(x - 1, nx), y, z), site(p->n, wrap(x + 1, nx), y, z),
                    site(p->n, x, wrap(y - 1, ny), z), site(p->n, x, wrap(y + 1, ny), z),
                    site(p->n, x, y, wrap(z - 1, nz)), site(p->n, x, y, wrap(z + 1, nz)),
                };
                for (int comp = 0; comp < 2; ++comp) {
                    double sum = 0.0;
                    for (int k = 0; k < 6; ++k) sum += phi[2 * nb[k] + comp];
                    double lap = (sum - 6.0 * phi[2 * s + comp]) * inv_dx2;
                    double mod2 = phi[2 * s] * phi[2 * s] + phi[2 * s + 1] * phi[2 * s + 1];
                    double force = lap - m * (mod2 - eta2) * phi[2 * s + comp];
                    pi[2 * s + comp] = ((1.0 - d) * pi[2 * s + comp] + dt * force) / (1.0 + d);
                }
            }
    /* pass 2: phi_{n+1} = phi_n + dt pi_{n+1/2} */
    const int64_t total = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < 2 * total; ++s) phi[s] += dt * pi[s];
}

/* nsteps leapfrog steps starting at level0. */
void or_run(const or_params *p, int64_t level0, int64_t nsteps, double *phi, double *pi, int nthreads)
{
    for (int64_t k = 0; k < nsteps; ++k) or_step(p, level0 + k, phi, pi, nthreads);
}

/*
 * The FP32-storage twin of or_run: the same FP64 steps, with phi and pi
 * rounded to FP32 (round to nearest) after every step.  Its distance from
 * or_run is the error that storing the field in FP32 costs by itself, the
 * floor of any scheme that keeps its state in FP32.
 */
void or_run_fp32_storage(const or_params *p, int64_t level0, int64_t nsteps, double *phi, double *pi, int nthreads)
{
    const int64_t n2 = 2 * (int64_t)p->n[0] * p->n[1] * p->n[2];
    for (int64_t k = 0; k < nsteps; ++k) {
        or_step(p, level0 + k, phi, pi, nthreads);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n2; ++i) {
            phi[i] = (double)(float)phi[i];
            pi[i] = (double)(float)pi[i];
        }
    }
}

/*
 * Energy of a stored state (phi_n, pi) at level n, split in its three terms:
 *   out[0] = sum |pi|^2
 *   out[1] = sum_i sum_x |phi(x + e_i) - phi(x)|^2 / dx^2
 *   out[2] = sum_x a_n^2 (lambda / 2) (|phi|^2 - eta^2)^2
 */
void or_energy_parts(const or_params *p, int64_t level, const double *phi, const double *pi,
                     double out[3], int nthreads)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    double co[6];
    or_level_coeffs(p, level, co);
    const double a = co[1];
    const double inv_dx2 = 1.0 / (p->dx * p->dx), eta2 = p->eta * p->eta;
    double kin = 0.0, grad = 0.0, pot = 0.0;
    set_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(+ : kin, grad, pot)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t s = site(p->n, x, y, z);
                int64_t fw[3] = {site(p->n, wrap(x + 1, nx), y, z), site(p->n, x, wrap(y + 1, ny), z),
                                 site(p->n, x, y, wrap(z + 1, nz))};
                kin += pi[2 * s] * pi[2 * s] + pi[2 * s + 1] * pi[2 * s + 1];
                for (int k = 0; k < 3; ++k) {
                    double dr = phi[2 * fw[k]] - phi[2 * s];
                    double di = phi[2 * fw[k] + 1] - phi[2 * s + 1];
                    grad += (dr * dr + di * di) * inv_dx2;
                }
                double mod2 = phi[2 * s] * phi[2 * s] + phi[2 * s + 1] * phi[2 * s + 1];
                pot += a * a * 0.5 * p->lambda * (mod2 - eta2) * (mod2 - eta2);
            }
    out[0] = kin;
    out[1] = grad;
    out[2] = pot;
}

/* Re sum_x conj(phi(x)) * (-Lap7 psi)(x) / dx^2 : the bilinear form of the
 * lattice Laplacian (used by the exactly conserved linear energy). */
double or_lap_dot(const int32_t n[3], double dx, const double *phi, const double *psi, int nthreads)
{
    const int nx = n[0], ny = n[1], nz = n[2];
    double acc = 0.0;
    set_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t s = site(n, x, y, z);
                int64_t nb[6] = {
                    site(n, wrap(x - 1, nx), y, z), site(n, wrap(x + 1, nx), y, z),
                    site(n, x, wrap(y - 1, ny), z), site(n, x, wrap(y + 1, ny), z),
                    site(n, x, y, wrap(z - 1, nz)), site(n, x, y, wrap(z + 1, nz)),
                };
                for (int comp = 0; comp < 2; ++comp) {
                    double sum = 0.0;
                    for (int k = 0; k < 6; ++k) sum += psi[2 * nb[k] + comp];
                    double neg_lap = (6.0 * psi[2 * s + comp] - sum) / (dx * dx);
                    acc += phi[2 * s + comp] * neg_lap;
                }
            }
    return acc;
}

/*
 * Winding number of the field around each lattice plaquette.
 *
 * The plaquette at site x normal to axis k has corners
 *     p0 = x, p1 = x + e_a, p2 = x + e_a + e_b, p3 = x + e_b,   (a, b) = (k+1, k+2) mod 3,
 * traversed counter-clockwise about +e_k.  Its winding is the winding number
 * about 0 of the closed polygon phi(p0) phi(p1) phi(p2) phi(p3) in the complex
 * plane, counted by signed crossings of the positive real axis:
 *   an edge u -> v crossing upward (Im u < 0 <= Im v) with cross(u, v) >= 0 adds +1,
 *   an edge u -> v crossing downward (Im v < 0 <= Im u) with cross(u, v) <= 0 adds -1,
 * where cross(u, v) = Re u Im v - Im u Re v.  A vertex on the axis counts as
 * above it; a chord through 0 counts as crossing the positive axis.  The
 * per-edge count is antisymmetric under reversing the edge, so the oriented
 * sum over the six faces of any cube is exactly zero.
 *
 * Inputs are FP32; the two products of cross() are exact in FP64 and the sign
 * of their FP64 difference is the sign of the exact difference, so the result
 * is exact.  Output w[k * sites + s] in {-4..4} (in practice -1, 0, 1).
 */
static int edge_crossing(const float *u, const float *v)
{
    double ur = u[0], ui = u[1], vr = v[0], vi = v[1];
    double cross = ur * vi - ui * vr;
    int u_above = ui >= 0.0, v_above = vi >= 0.0;
    if (!u_above && v_above) return cross >= 0.0 ? 1 : 0;
    if (u_above && !v_above) return cross <= 0.0 ? -1 : 0;
    return 0;
}

void or_winding(const int32_t n[3], const float *phi, int8_t *w, int nthreads)
{
    const int nx = n[0], ny = n[1], nz = n[2];
    const int64_t sites = (int64_t)nx * ny * nz;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c[3] = {x, y, z};
                for (int k = 0; k < 3; ++k) {
                    int a = (k + 1) % 3, b = (k + 2) % 3;
                    int q[4][3];
                    for (int i = 0; i < 4; ++i) memcpy(q[i], c, sizeof c);
                    q[1][a] = wrap(q[1][a] + 1, n[a]);
                    q[2][a] = wrap(q[2][a] + 1, n[a]);
                    q[2][b] = wrap(q[2][b] + 1, n[b]);
                    q[3][b] = wrap(q[3][b] + 1, n[b]);
                    int total = 0;
                    for (int i = 0; i < 4; ++i) {
                        const float *u = phi + 2 * site(n, q[i][0], q[i][1], q[i][2]);
                        const float *v = phi + 2 * site(n, q[(i + 1) % 4][0], q[(i + 1) % 4][1], q[(i + 1) % 4][2]);
                        total += edge_crossing(u, v);
                    }
                    w[k * sites + site(n, x, y, z)] = (int8_t)total;
                }
            }
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
