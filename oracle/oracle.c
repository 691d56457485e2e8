/*
 * oracle.c -- plain FP64 CPU oracle for the stencil engine.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU
 * baseline call this file through oracle/__init__.py.  The library never links, loads or
 * calls it, and it shares no code, header, table or helper with the CUDA path.
 *
 * Everything here is the plain definition, evaluated naively in double precision and built
 * with -ffp-contract=off so that no multiply-add is fused:
 *
 *   beta, f^   the augmented (padded) array of Eq. 2, with a periodic boundary function:
 *              the halo of width r holds the periodic image of the interior (Sec. 2.4).
 *   zeta       the discrete cross-correlation f'_i = sum_{j=-r..r} g_j f^_{i+j}, Eq. 3
 *              (Sec. 3.1).
 *   maxfilter  the nonlinear 1D stencil f'_i = max_{j=-r..r} f^_{i+j} (max filtering, Sec. 2.1),
 *              evaluated as the plain maximum over each window.
 *   diffusion  one forward-Euler step of df/dt = alpha lap f, Eq. 4 (Sec. 3.2), evaluated
 *              literally as f + dt*alpha*(sum over axes of the 2nd-derivative stencil); the
 *              folded single-kernel form of Eqs. 5-7 is the CUDA path's business, not ours.
 *   diffusion_r  the same step with the radius-r central 2nd derivative of order 2r (the
 *              radius sweep of Sec. 5.3, r = 1..4, in 1, 2 or 3 dimensions).  The weights are
 *              the classical maximal-order central ones, evaluated from their closed form
 *              c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), k = 1..r, c_0 = -2 sum 1/k^2.
 *   derivs     6th-order central differences (Sec. 3.3 names the order; the weights are the
 *              textbook ones: 1st derivative (-1,9,-45,0,45,-9,1)/60, 2nd derivative
 *              (2,-27,270,-490,270,-27,2)/180, and the mixed derivative in the diagonal form
 *              [270 D(1) - 27 D(2) + 2 D(3)] / (720 dx dy) with
 *              D(a) = f(a,a) - f(a,-a) + f(-a,-a) - f(-a,a)).
 *   mhd_rhs    the right-hand side of the non-ideal MHD equations A1-A4 (Appendix A,
 *              Table A1), with heating and cooling switched off (H = C = 0).  The conduction
 *              term div(K grad T) of A3 takes a constant K and is evaluated through the
 *              identity T = T0 exp(phi), phi = gamma s/cp + (gamma-1)(lnrho - lnrho0):
 *              div(K grad T) / (rho T) = (K / rho) (lap phi + |grad phi|^2), with the
 *              6th-order derivatives of lnrho and s.
 *   rk3        the 3-stage explicit Runge-Kutta step of Sec. 3.3.  The paper does not print
 *              its coefficients; the reading taken is Williamson's 2N-storage 3rd-order
 *              scheme: w <- alpha_s w + dt RHS(f); f <- f + beta_s w, with
 *              alpha = (0, -5/9, -153/128) and beta = (1/3, 15/16, 8/15).
 *
 * Layout (the oracle's own): a padded "box" is a dense array of extents
 * (nx+2r) x (ny+2r) x (nz+2r), x fastest; an axis of interior extent 1 gets no halo.
 * Interior arrays are dense (nz, ny, nx).
 *
 * Parity: every function is pinned by tests that do not use this file's arithmetic
 * (closed forms, polynomial exactness, library routines, brute force); see tests/.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define R 3 /* radius of the 6th-order central differences */

/* ------------------------------------------------------------------ padding (Eq. 2) */

static int64_t halo_of(int64_t n, int r) { return n > 1 ? r : 0; }

static int64_t wrap(int64_t i, int64_t n) {
    int64_t m = i % n;
    return m < 0 ? m + n : m;
}

/* f^ with periodic beta: every cell of the padded box takes the value of interior cell
 * ((i - h) mod n) along each axis. Works for any element size. */
static void pad_periodic(const void *interior, int64_t nx, int64_t ny, int64_t nz, int r,
                         size_t esize, void *padded) {
    int64_t hx = halo_of(nx, r), hy = halo_of(ny, r), hz = halo_of(nz, r);
    int64_t px = nx + 2 * hx, py = ny + 2 * hy, pz = nz + 2 * hz;
    const char *src = (const char *)interior;
    char *dst = (char *)padded;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < pz; ++k)
        for (int64_t j = 0; j < py; ++j)
            for (int64_t i = 0; i < px; ++i) {
                int64_t si = wrap(i - hx, nx), sj = wrap(j - hy, ny), sk = wrap(k - hz, nz);
                memcpy(dst + ((k * py + j) * px + i) * esize,
                       src + ((sk * ny + sj) * nx + si) * esize, esize);
            }
}

void oracle_pad_periodic_f64(const double *in, int64_t nx, int64_t ny, int64_t nz, int r,
                             double *out) {
    pad_periodic(in, nx, ny, nz, r, sizeof(double), out);
}

/* ------------------------------------------------------- cross-correlation (Eq. 3) */

/* One sweep over a padded 1D array fhat[n + 2r]; out[n] is the interior result. */
void oracle_xcorr1d_box_f64(const double *fhat, int64_t n, const double *g, int r,
                            double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = -r; j <= r; ++j) acc += g[j + r] * fhat[i + r + j];
        out[i] = acc;
    }
}

/* Integer variant: arithmetic modulo 2^32 (two's-complement wraparound), done in uint32. */
void oracle_xcorr1d_box_u32(const uint32_t *fhat, int64_t n, const int32_t *g, int r,
                            uint32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t acc = 0u;
        for (int j = -r; j <= r; ++j) acc += (uint32_t)g[j + r] * fhat[i + r + j];
        out[i] = acc;
    }
}

/* `sweeps` periodic sweeps, each feeding the next: pad (Eq. 2), correlate (Eq. 3). */
int oracle_xcorr1d_f64(const double *in, int64_t n, const double *g, int r, int sweeps,
                       double *out) {
    double *cur = malloc(sizeof(double) * n), *hat = malloc(sizeof(double) * (n + 2 * r));
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(double) * n);
    for (int s = 0; s < sweeps; ++s) {
        pad_periodic(cur, n, 1, 1, r, sizeof(double), hat);
        oracle_xcorr1d_box_f64(hat, n, g, r, cur);
    }
    memcpy(out, cur, sizeof(double) * n);
    free(cur); free(hat);
    return 0;
}

int oracle_xcorr1d_u32(const uint32_t *in, int64_t n, const int32_t *g, int r, int sweeps,
                       uint32_t *out) {
    uint32_t *cur = malloc(sizeof(uint32_t) * n), *hat = malloc(sizeof(uint32_t) * (n + 2 * r));
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(uint32_t) * n);
    for (int s = 0; s < sweeps; ++s) {
        pad_periodic(cur, n, 1, 1, r, sizeof(uint32_t), hat);
        oracle_xcorr1d_box_u32(hat, n, g, r, cur);
    }
    memcpy(out, cur, sizeof(uint32_t) * n);
    free(cur); free(hat);
    return 0;
}

/* ------------------------------------------ max filtering (nonlinear stencil, Sec. 2.1) */

void oracle_maxfilter1d_box_f64(const double *fhat, int64_t n, int r, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double m = fhat[i];
        for (int j = 1; j <= 2 * r; ++j)
            if (fhat[i + j] > m) m = fhat[i + j];
        out[i] = m;
    }
}

void oracle_maxfilter1d_box_i32(const int32_t *fhat, int64_t n, int r, int32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t m = fhat[i];
        for (int j = 1; j <= 2 * r; ++j)
            if (fhat[i + j] > m) m = fhat[i + j];
        out[i] = m;
    }
}

/* `sweeps` periodic max-filter sweeps, each feeding the next. */
int oracle_maxfilter1d_f64(const double *in, int64_t n, int r, int sweeps, double *out) {
    double *cur = malloc(sizeof(double) * n), *hat = malloc(sizeof(double) * (n + 2 * r));
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(double) * n);
    for (int s = 0; s < sweeps; ++s) {
        pad_periodic(cur, n, 1, 1, r, sizeof(double), hat);
        oracle_maxfilter1d_box_f64(hat, n, r, cur);
    }
    memcpy(out, cur, sizeof(double) * n);
    free(cur); free(hat);
    return 0;
}

int oracle_maxfilter1d_i32(const int32_t *in, int64_t n, int r, int sweeps, int32_t *out) {
    int32_t *cur = malloc(sizeof(int32_t) * n), *hat = malloc(sizeof(int32_t) * (n + 2 * r));
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(int32_t) * n);
    for (int s = 0; s < sweeps; ++s) {
        pad_periodic(cur, n, 1, 1, r, sizeof(int32_t), hat);
        oracle_maxfilter1d_box_i32(hat, n, r, cur);
    }
    memcpy(out, cur, sizeof(int32_t) * n);
    free(cur); free(hat);
    return 0;
}

/* ------------------------------------------------- 6th-order central differences */

static const double C1[7] = {-1.0 / 60.0, 3.0 / 20.0, -3.0 / 4.0, 0.0,
                             3.0 / 4.0,   -3.0 / 20.0, 1.0 / 60.0};
static const double C2[7] = {1.0 / 90.0, -3.0 / 20.0, 3.0 / 2.0, -49.0 / 18.0,
                             3.0 / 2.0,  -3.0 / 20.0, 1.0 / 90.0};
static const double CM[3] = {270.0, -27.0, 2.0}; /* mixed, offsets a = 1, 2, 3; / 720 */

/* d/dx along a stride s at linear index p of a padded box, spacing h. */
static double der1(const double *f, int64_t p, int64_t s, double h) {
    double acc = 0.0;
    for (int j = -R; j <= R; ++j) acc += C1[j + R] * f[p + j * s];
    return acc / h;
}

static double der2(const double *f, int64_t p, int64_t s, double h) {
    double acc = 0.0;
    for (int j = -R; j <= R; ++j) acc += C2[j + R] * f[p + j * s];
    return acc / (h * h);
}

static double dermix(const double *f, int64_t p, int64_t s1, int64_t s2, double h1, double h2) {
    double acc = 0.0;
    for (int a = 1; a <= R; ++a) {
        double d = f[p + a * s1 + a * s2] - f[p + a * s1 - a * s2] + f[p - a * s1 - a * s2] -
                   f[p - a * s1 + a * s2];
        acc += CM[a - 1] * d;
    }
    return acc / (720.0 * h1 * h2);
}

/* All derivatives at every interior cell of a padded 3D box (halo R on each axis).
 * out has 9 planes of nx*ny*nz values: dx, dy, dz, dxx, dyy, dzz, dxy, dxz, dyz. */
void oracle_derivs_box(const double *fhat, int64_t nx, int64_t ny, int64_t nz,
                       const double *h, double *out) {
    int64_t px = nx + 2 * R, py = ny + 2 * R, sx = 1, sy = px, sz = px * py;
    int64_t ncell = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = ((k + R) * py + (j + R)) * px + (i + R), o = (k * ny + j) * nx + i;
                out[0 * ncell + o] = der1(fhat, p, sx, h[0]);
                out[1 * ncell + o] = der1(fhat, p, sy, h[1]);
                out[2 * ncell + o] = der1(fhat, p, sz, h[2]);
                out[3 * ncell + o] = der2(fhat, p, sx, h[0]);
                out[4 * ncell + o] = der2(fhat, p, sy, h[1]);
                out[5 * ncell + o] = der2(fhat, p, sz, h[2]);
                out[6 * ncell + o] = dermix(fhat, p, sx, sy, h[0], h[1]);
                out[7 * ncell + o] = dermix(fhat, p, sx, sz, h[0], h[2]);
                out[8 * ncell + o] = dermix(fhat, p, sy, sz, h[1], h[2]);
            }
}

/* ------------------------------------------------------- diffusion (Eq. 4, Sec. 3.2) */

/* One forward-Euler step f' = f + dt*alpha*lap f over a padded box of `ndim` dimensions
 * (axes of extent 1 have no halo and contribute no 2nd derivative). out is the interior. */
void oracle_diffusion_box(const double *fhat, int64_t nx, int64_t ny, int64_t nz,
                          double dt, double alpha, const double *h, double *out) {
    int64_t hx = halo_of(nx, R), hy = halo_of(ny, R), hz = halo_of(nz, R);
    int64_t px = nx + 2 * hx, py = ny + 2 * hy;
    int64_t n[3] = {nx, ny, nz}, s[3] = {1, px, px * py};
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = ((k + hz) * py + (j + hy)) * px + (i + hx);
                double lap = 0.0;
                for (int a = 0; a < 3; ++a)
                    if (n[a] > 1) lap += der2(fhat, p, s[a], h[a]);
                out[(k * ny + j) * nx + i] = fhat[p] + dt * alpha * lap;
            }
}

/* `steps` periodic Euler steps of the diffusion equation; in/out are dense interiors. */
int oracle_diffusion(const double *in, int64_t nx, int64_t ny, int64_t nz, double dt,
                     double alpha, const double *h, int steps, double *out) {
    int64_t hx = halo_of(nx, R), hy = halo_of(ny, R), hz = halo_of(nz, R);
    size_t ncell = (size_t)(nx * ny * nz);
    size_t npad = (size_t)((nx + 2 * hx) * (ny + 2 * hy) * (nz + 2 * hz));
    double *cur = malloc(sizeof(double) * ncell), *hat = malloc(sizeof(double) * npad);
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(double) * ncell);
    for (int t = 0; t < steps; ++t) {
        pad_periodic(cur, nx, ny, nz, R, sizeof(double), hat);
        oracle_diffusion_box(hat, nx, ny, nz, dt, alpha, h, cur);
    }
    memcpy(out, cur, sizeof(double) * ncell);
    free(cur); free(hat);
    return 0;
}

/* ------------------------------------ radius-r diffusion (Eq. 4, radius sweep, Sec. 5.3) */

#define RMAX 4

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Weights of the order-2r central second derivative on points -r..r (unit spacing):
 * c[0] is the centre weight, c[k] the weight of each of the points at +-k. */
static void d2_weights(int r, double *c) {
    double centre = 0.0;
    for (int k = 1; k <= r; ++k) {
        double sign = (k % 2 == 1) ? 1.0 : -1.0;
        c[k] = 2.0 * sign * factorial(r) * factorial(r) /
               ((double)k * (double)k * factorial(r - k) * factorial(r + k));
        centre += 1.0 / ((double)k * (double)k);
    }
    c[0] = -2.0 * centre;
}

static double der2_r(const double *f, int64_t p, int64_t s, double h, int r, const double *c) {
    double acc = c[0] * f[p];
    for (int k = 1; k <= r; ++k) acc += c[k] * (f[p + k * s] + f[p - k * s]);
    return acc / (h * h);
}

/* One forward-Euler step f' = f + dt*alpha*lap f with the radius-r Laplacian over a padded
 * box (halo r on every axis of extent > 1).  Returns -1 for r outside 1..RMAX. */
int oracle_diffusion_r_box(const double *fhat, int64_t nx, int64_t ny, int64_t nz, int r,
                           double dt, double alpha, const double *h, double *out) {
    if (r < 1 || r > RMAX) return -1;
    double c[RMAX + 1];
    d2_weights(r, c);
    int64_t hx = halo_of(nx, r), hy = halo_of(ny, r), hz = halo_of(nz, r);
    int64_t px = nx + 2 * hx, py = ny + 2 * hy;
    int64_t n[3] = {nx, ny, nz}, s[3] = {1, px, px * py};
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                int64_t p = ((k + hz) * py + (j + hy)) * px + (i + hx);
                double lap = 0.0;
                for (int a = 0; a < 3; ++a)
                    if (n[a] > 1) lap += der2_r(fhat, p, s[a], h[a], r, c);
                out[(k * ny + j) * nx + i] = fhat[p] + dt * alpha * lap;
            }
    return 0;
}

/* `steps` periodic Euler steps with the radius-r Laplacian; in/out are dense interiors. */
int oracle_diffusion_r(const double *in, int64_t nx, int64_t ny, int64_t nz, int r, double dt,
                       double alpha, const double *h, int steps, double *out) {
    if (r < 1 || r > RMAX) return -1;
    int64_t hx = halo_of(nx, r), hy = halo_of(ny, r), hz = halo_of(nz, r);
    size_t ncell = (size_t)(nx * ny * nz);
    size_t npad = (size_t)((nx + 2 * hx) * (ny + 2 * hy) * (nz + 2 * hz));
    double *cur = malloc(sizeof(double) * ncell), *hat = malloc(sizeof(double) * npad);
    if (!cur || !hat) { free(cur); free(hat); return -1; }
    memcpy(cur, in, sizeof(double) * ncell);
    for (int t = 0; t < steps; ++t) {
        pad_periodic(cur, nx, ny, nz, r, sizeof(double), hat);
        oracle_diffusion_r_box(hat, nx, ny, nz, r, dt, alpha, h, cur);
    }
    memcpy(out, cur, sizeof(double) * ncell);
    free(cur); free(hat);
    return 0;
}

/* ------------------------------------------------------ MHD right-hand side (App. A) */

/* Field order of the state: */
enum { LNRHO = 0, UX, UY, UZ, AX, AY, AZ, SS, NF };

/* Physical parameters, passed as an array so no struct crosses the ABI:
 * par[0..2] = dx, dy, dz; par[3] = cs0; par[4] = gamma; par[5] = cp; par[6] = lnrho0;
 * par[7] = nu; par[8] = eta; par[9] = zeta; par[10] = mu0; par[11] = K (heat conductivity). */
enum { P_DX = 0, P_DY, P_DZ, P_CS0, P_GAMMA, P_CP, P_LNRHO0, P_NU, P_ETA, P_ZETA, P_MU0, P_K, NPAR };

/* RHS of Eqs. A1-A4 at every interior cell of 8 padded boxes (halo R), written to rhs[f]
 * (dense interiors). fhat[f] and rhs[f] are separate arrays per field. */
void oracle_mhd_rhs_box(const double *const *fhat, int64_t nx, int64_t ny, int64_t nz,
                        const double *par, double *const *rhs) {
    const int64_t px = nx + 2 * R, py = ny + 2 * R;
    const int64_t st[3] = {1, px, px * py};
    const double h[3] = {par[P_DX], par[P_DY], par[P_DZ]};
    const double cs0 = par[P_CS0], gam = par[P_GAMMA], cp = par[P_CP], lnrho0 = par[P_LNRHO0];
    const double nu = par[P_NU], eta = par[P_ETA], zeta = par[P_ZETA], mu0 = par[P_MU0];
    const double K = par[P_K];
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i) {
                const int64_t p = ((k + R) * py + (j + R)) * px + (i + R);
                const int64_t o = (k * ny + j) * nx + i;
                /* values */
                double lnrho = fhat[LNRHO][p], ss = fhat[SS][p];
                double u[3] = {fhat[UX][p], fhat[UY][p], fhat[UZ][p]};
                /* first derivatives: grad lnrho, grad s, du[i][a] = d u_i / d x_a, dA likewise */
                double glnrho[3], gss[3], du[3][3], dA[3][3];
                for (int a = 0; a < 3; ++a) {
                    glnrho[a] = der1(fhat[LNRHO], p, st[a], h[a]);
                    gss[a] = der1(fhat[SS], p, st[a], h[a]);
                    for (int c = 0; c < 3; ++c) {
                        du[c][a] = der1(fhat[UX + c], p, st[a], h[a]);
                        dA[c][a] = der1(fhat[AX + c], p, st[a], h[a]);
                    }
                }
                /* second derivatives: Hu[i][a][b] = d^2 u_i / dx_a dx_b (symmetric), HA likewise */
                double Hu[3][3][3], HA[3][3][3];
                for (int c = 0; c < 3; ++c)
                    for (int a = 0; a < 3; ++a)
                        for (int b = a; b < 3; ++b) {
                            double vu, vA;
                            if (a == b) {
                                vu = der2(fhat[UX + c], p, st[a], h[a]);
                                vA = der2(fhat[AX + c], p, st[a], h[a]);
                            } else {
                                vu = dermix(fhat[UX + c], p, st[a], st[b], h[a], h[b]);
                                vA = dermix(fhat[AX + c], p, st[a], st[b], h[a], h[b]);
                            }
                            Hu[c][a][b] = Hu[c][b][a] = vu;
                            HA[c][a][b] = HA[c][b][a] = vA;
                        }
                /* derived quantities (Table A1) */
                double divu = du[0][0] + du[1][1] + du[2][2];
                double lapu[3], graddivu[3], lapA[3], graddivA[3];
                for (int c = 0; c < 3; ++c) {
                    lapu[c] = Hu[c][0][0] + Hu[c][1][1] + Hu[c][2][2];
                    lapA[c] = HA[c][0][0] + HA[c][1][1] + HA[c][2][2];
                    graddivu[c] = Hu[0][c][0] + Hu[1][c][1] + Hu[2][c][2];
                    graddivA[c] = HA[0][c][0] + HA[1][c][1] + HA[2][c][2];
                }
                /* traceless rate-of-shear S_ab = (du_a/dx_b + du_b/dx_a)/2 - delta_ab div u / 3 */
                double S[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        S[a][b] = 0.5 * (du[a][b] + du[b][a]) - (a == b ? divu / 3.0 : 0.0);
                /* B = curl A; j = curl B / mu0 = (grad div A - lap A) / mu0 */
                double B[3] = {dA[2][1] - dA[1][2], dA[0][2] - dA[2][0], dA[1][0] - dA[0][1]};
                double jj[3];
                for (int c = 0; c < 3; ++c) jj[c] = (graddivA[c] - lapA[c]) / mu0;
                double jxB[3] = {jj[1] * B[2] - jj[2] * B[1], jj[2] * B[0] - jj[0] * B[2],
                                 jj[0] * B[1] - jj[1] * B[0]};
                double uxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2],
                                 u[0] * B[1] - u[1] * B[0]};
                /* ideal-gas closure */
                double rho = exp(lnrho);
                double cs2 = cs0 * cs0 * exp(gam * ss / cp + (gam - 1.0) * (lnrho - lnrho0));
                double TT = cs2 / (cp * (gam - 1.0));
                /* A1: D lnrho / Dt = -div u */
                double ugradlnrho = u[0] * glnrho[0] + u[1] * glnrho[1] + u[2] * glnrho[2];
                rhs[LNRHO][o] = -ugradlnrho - divu;
                /* A2: Du/Dt = -cs2 grad(s/cp + lnrho) + jxB/rho
                 *             + nu (lap u + grad div u / 3 + 2 S.grad lnrho) + zeta grad div u */
                for (int c = 0; c < 3; ++c) {
                    double adv = u[0] * du[c][0] + u[1] * du[c][1] + u[2] * du[c][2];
                    double Sg = S[c][0] * glnrho[0] + S[c][1] * glnrho[1] + S[c][2] * glnrho[2];
                    rhs[UX + c][o] = -adv - cs2 * (gss[c] / cp + glnrho[c]) + jxB[c] / rho +
                                     nu * (lapu[c] + graddivu[c] / 3.0 + 2.0 * Sg) +
                                     zeta * graddivu[c];
                }
                /* A3: rho T Ds/Dt = div(K grad T) + eta mu0 j^2 + 2 rho nu S:S + zeta rho (div u)^2
                 * (H = C = 0) */
                double j2 = jj[0] * jj[0] + jj[1] * jj[1] + jj[2] * jj[2];
                double SS2 = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) SS2 += S[a][b] * S[a][b];
                double ugrads = u[0] * gss[0] + u[1] * gss[1] + u[2] * gss[2];
                rhs[SS][o] = -ugrads + (eta * mu0 * j2 + 2.0 * rho * nu * SS2 +
                                        zeta * rho * divu * divu) / (rho * TT);
                if (K != 0.0) {
                    /* div(K grad T) / (rho T) with T = T0 exp(phi): (K / rho)(lap phi + |grad phi|^2) */
                    double lapphi = 0.0, gphi2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double gphi = gam / cp * gss[a] + (gam - 1.0) * glnrho[a];
                        gphi2 += gphi * gphi;
                        lapphi += gam / cp * der2(fhat[SS], p, st[a], h[a]) +
                                  (gam - 1.0) * der2(fhat[LNRHO], p, st[a], h[a]);
                    }
                    rhs[SS][o] += K / rho * (lapphi + gphi2);
                }
                /* A4: dA/dt = u x B + eta lap A */
                for (int c = 0; c < 3; ++c) rhs[AX + c][o] = uxB[c] + eta * lapA[c];
            }
}

/* --------------------------------------------------------------- RK3 (Sec. 3.3) */

static const double RK_ALPHA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_BETA[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

/* `steps` periodic RK3 steps of the MHD system. f[NF * ncell] (dense interiors, field-major)
 * is advanced in place. */
int oracle_mhd_rk3(double *f, int64_t nx, int64_t ny, int64_t nz, const double *par, double dt,
                   int steps) {
    size_t ncell = (size_t)(nx * ny * nz);
    size_t npad = (size_t)((nx + 2 * R) * (ny + 2 * R) * (nz + 2 * R));
    double *hat = malloc(sizeof(double) * npad * NF);
    double *rhs = malloc(sizeof(double) * ncell * NF);
    double *w = calloc(ncell * NF, sizeof(double));
    if (!hat || !rhs || !w) { free(hat); free(rhs); free(w); return -1; }
    const double *hp[NF];
    double *rp[NF];
    for (int q = 0; q < NF; ++q) { hp[q] = hat + q * npad; rp[q] = rhs + q * ncell; }
    for (int t = 0; t < steps; ++t)
        for (int s = 0; s < 3; ++s) {
            for (int q = 0; q < NF; ++q)
                pad_periodic(f + q * ncell, nx, ny, nz, R, sizeof(double), hat + q * npad);
            oracle_mhd_rhs_box(hp, nx, ny, nz, par, rp);
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < (int64_t)(ncell * NF); ++c) {
                w[c] = RK_ALPHA[s] * w[c] + dt * rhs[c];
                f[c] = f[c] + RK_BETA[s] * w[c];
            }
        }
    free(hat); free(rhs); free(w);
    return 0;
}

/* One RK3 step on a NON-periodic box, for checking single output cells of a large grid:
 * f[NF * m^3 dense, extents (mx, my, mz)] holds a neighbourhood cut out of the periodic grid.
 * Each substep only updates cells with a full radius-R neighbourhood inside the region still
 * valid, so after `nsub` substeps the valid region is the box shrunk by R*nsub on every side.
 * On return f holds the advanced values there (and stale values elsewhere). */
int oracle_mhd_rk3_box(double *f, int64_t mx, int64_t my, int64_t mz, const double *par,
                       double dt, int nsub) {
    size_t ncell = (size_t)(mx * my * mz);
    double *w = calloc(ncell * NF, sizeof(double));
    double *rhs = malloc(sizeof(double) * ncell * NF);
    double *box = malloc(sizeof(double) * ncell * NF);
    if (!w || !rhs || !box) { free(w); free(rhs); free(box); return -1; }
    for (int s = 0; s < nsub; ++s) {
        int64_t lo = (int64_t)R * s; /* valid input region is [lo, m - lo) */
        int64_t nx = mx - 2 * (lo + R), ny = my - 2 * (lo + R), nz = mz - 2 * (lo + R);
        if (nx <= 0 || ny <= 0 || nz <= 0) { free(w); free(rhs); free(box); return -2; }
        int64_t bx = nx + 2 * R, by = ny + 2 * R, bz = nz + 2 * R;
        const double *hp[NF];
        double *rp[NF];
        for (int q = 0; q < NF; ++q) {
            double *bq = box + q * ncell;
            for (int64_t k = 0; k < bz; ++k)
                for (int64_t j = 0; j < by; ++j)
                    for (int64_t i = 0; i < bx; ++i)
                        bq[(k * by + j) * bx + i] =
                            f[q * ncell + ((k + lo) * my + (j + lo)) * mx + (i + lo)];
            hp[q] = bq;
            rp[q] = rhs + q * ncell;
        }
        oracle_mhd_rhs_box(hp, nx, ny, nz, par, rp);
        for (int q = 0; q < NF; ++q)
            for (int64_t k = 0; k < nz; ++k)
                for (int64_t j = 0; j < ny; ++j)
                    for (int64_t i = 0; i < nx; ++i) {
                        size_t c = q * ncell + ((k + lo + R) * my + (j + lo + R)) * mx + (i + lo + R);
                        double r = rhs[q * ncell + (k * ny + j) * nx + i];
                        w[c] = RK_ALPHA[s] * w[c] + dt * r;
                        f[c] = f[c] + RK_BETA[s] * w[c];
                    }
    }
    free(w); free(rhs); free(box);
    return 0;
}

/* ------------------------------------------------------------------------- norms */

/* out = {sum f, sum f^2, max |f|} over n values, accumulated in long double. */
void oracle_norms(const double *f, int64_t n, double *out) {
    long double s = 0.0L, s2 = 0.0L;
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        s += f[i];
        s2 += (long double)f[i] * f[i];
        double a = fabs(f[i]);
        if (a > m) m = a;
    }
    out[0] = (double)s;
    out[1] = (double)s2;
    out[2] = m;
}

/* sum exp(lnrho) over n values (the mass, up to the cell volume), in long double. */
double oracle_mass(const double *lnrho, int64_t n) {
    long double s = 0.0L;
    for (int64_t i = 0; i < n; ++i) s += exp(lnrho[i]);
    return (double)s;
}
