/*
 * se2ot_oracle.c -- FP64 CPU oracle for the SE(2) Gibbs-kernel group convolution and
 * the convolutional Sinkhorn barycenter of "Optimal Transport on the Lie Group of
 * Roto-translations" (arXiv 2402.15322).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, with the passage each function follows:
 *   or_group_mul / or_group_inv  -- SE(2) product and inverse in fixed coordinates
 *                                   (x, y, theta), Sec. 2.3 (group law, small-angle
 *                                   convention theta in [-pi, pi)).
 *   or_rho_b2                    -- squared half-angle distance rho_b^2, Sec. 4.3,
 *                                   Eq. (rho_b) with the half-angle coordinates b^1..b^3.
 *   or_rho_c2                    -- squared logarithmic distance rho_c^2 = ||log g||^2, Sec. 4.3,
 *                                   with the SE(2) logarithm from inverting the exponential map.
 *                                   Every kernel function takes `dist`: 0 rho_b, 1 rho_c.
 *   or_log_kernel                -- log K(h^-1 g) = -rho(h^-1 g)^2 / eps, the Gibbs kernel
 *                                   of Sec. 4.2 with p = 2 and d replaced by rho_b
 *                                   (Appendix A, kernel construction).
 *   or_taps                      -- the same kernel tabulated over the (2r+1)^2 spatial
 *                                   offsets and all orientation pairs of the grid.
 *   or_conv_lin                  -- (K * f)(g) = sum_h K(h^-1 g) f(h), Sec. 4.2, as a
 *                                   plain triple loop (uniform Haar weights, Sec. 2.3).
 *   or_conv_log                  -- log (K * exp(lf)), the same sum in the log domain with
 *                                   a per-output max shift (exact algebra); or_conv_log_points
 *                                   evaluates it at selected outputs only.
 *   or_barycenter_lin            -- Appendix A algorithm, literally, in the linear domain.
 *   or_barycenter_log            -- Appendix A algorithm with every scaling vector kept as
 *                                   its logarithm (same steps, same order).
 *   or_cost_taps                 -- log(c K) with c = rho_b^2: the kernel weighted by the cost,
 *                                   whose convolution gives the transport cost of a plan.
 *   or_prox_log / or_jko_log     -- entropic JKO steps of the porous-medium energy
 *                                   F = sum mu^m / (m - 1) (Sec. 2.2 Eq. (GF_JKO), Sec. 6.4):
 *                                   the scaling iterations of Sec. 4.1 with the marginal
 *                                   constraint on the first marginal and the KL-proximal map of
 *                                   tau F on the second, derived in or_prox_log.
 *   or_w2_log                    -- entropic transport between two measures, Sec. 4.1: the
 *                                   scaling iterations with the marginal-constraint prox
 *                                   (a = mu / K b, b = nu / K a), in the log domain, and the
 *                                   cost <c, pi> of the plan pi = a K b (Eq. (L^{W_p}), p = 2).
 *
 * Grid and layout.  Voxel (ix, iy, k) of an Nx x Ny x Nth grid stands for the group element
 * (ix/Nx, iy/Ny, 2 pi k/Nth).  Arrays are f[((b*Ny + y)*Nx + x)*Nth + k] (orientation
 * innermost).  The kernel is truncated to spatial offsets |dx|, |dy| <= r with every
 * orientation pair coupled.  Outside the grid the sum has no term (zero boundary) unless
 * `periodic` is set, in which case spatial indices wrap.
 *
 * Readings of the paper used here (the paper fixes none of them):
 *   - theta differences are wrapped to [-pi, pi); a difference of exactly pi maps to -pi.
 *   - no voxel-volume or Haar normalisation constant multiplies the kernel.
 *   - weights lambda_i == 0 contribute nothing to the geometric mean (0 * log d is skipped).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double OR_PI = 3.14159265358979323846264338327950288;

/* theta wrapped to the small-angle convention [-pi, pi). */
static double or_wrap(double th)
{
    double t = fmod(th + OR_PI, 2.0 * OR_PI);
    if (t < 0.0) t += 2.0 * OR_PI;
    return t - OR_PI;
}

int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The group law of Sec. 2.3:
 * (x,y,th)(x',y',th') = (x + x' cos th - y' sin th, y + x' sin th + y' cos th, th + th'). */
void or_group_mul(const double *a, const double *b, double *c)
{
    double ca = cos(a[2]), sa = sin(a[2]);
    double x = a[0] + b[0] * ca - b[1] * sa;
    double y = a[1] + b[0] * sa + b[1] * ca;
    double t = or_wrap(a[2] + b[2]);
    c[0] = x; c[1] = y; c[2] = t;
}

/* The inverse of Sec. 2.3: g^-1 = (-R^-1 x, R^-1). */
void or_group_inv(const double *a, double *c)
{
    double ca = cos(a[2]), sa = sin(a[2]);
    /* R^-1 = R(-th): (x, y) -> (x cos th + y sin th, -x sin th + y cos th) */
    double x = -(a[0] * ca + a[1] * sa);
    double y = -(-a[0] * sa + a[1] * ca);
    c[0] = x; c[1] = y; c[2] = or_wrap(-a[2]);
}

/* Sec. 4.3 Eq. (rho_b): rho_b(g)^2 = (w1 b1)^2 + (w2 b2)^2 + (w3 b3)^2 with the half-angle coordinates
 * b1 = x cos(th/2) + y sin(th/2), b2 = -x sin(th/2) + y cos(th/2), b3 = th, th in [-pi, pi). */
double or_rho_b2(double x, double y, double th, double w1, double w2, double w3)
{
    double t = or_wrap(th);
    double ch = cos(0.5 * t), sh = sin(0.5 * t);
    double b1 = x * ch + y * sh;
    double b2 = -x * sh + y * ch;
    double b3 = t;
    return (w1 * b1) * (w1 * b1) + (w2 * b2) * (w2 * b2) + (w3 * b3) * (w3 * b3);
}

/* rho_c(g)^2 = ||log g||^2 in the left-invariant metric diag(w1^2, w2^2, w3^2) on the basis
 * (A1, A2, A3) (Sec. 4.3, the logarithmic approximation).  The logarithm inverts the
 * exponential map exp(c1 A1 + c2 A2 + c3 A3) = (V(c3) (c1, c2), c3) with
 * V(t) = [[sin t / t, -(1 - cos t) / t], [(1 - cos t) / t, sin t / t]] (V(0) = identity):
 * c3 = th in [-pi, pi) and (c1, c2) solves the 2x2 system V(th) (c1, c2) = (x, y). */
double or_rho_c2(double x, double y, double th, double w1, double w2, double w3)
{
    double t = or_wrap(th);
    double p, q;   /* V = [[p, -q], [q, p]] */
    if (fabs(t) < 1e-8) {
        p = 1.0 - t * t / 6.0;
        q = t / 2.0;
    } else {
        p = sin(t) / t;
        q = (1.0 - cos(t)) / t;
    }
    double det = p * p + q * q;
    double c1 = (p * x + q * y) / det;
    double c2 = (-q * x + p * y) / det;
    return (w1 * c1) * (w1 * c1) + (w2 * c2) * (w2 * c2) + (w3 * t) * (w3 * t);
}

/* The squared distance the kernel uses: dist 0 = rho_b (the paper's choice), 1 = rho_c. */
double or_rho2(double x, double y, double th, double w1, double w2, double w3, int dist)
{
    return dist == 1 ? or_rho_c2(x, y, th, w1, w2, w3) : or_rho_b2(x, y, th, w1, w2, w3);
}

/* The Gibbs kernel of Sec. 4.2: log K(h^-1 g) = -rho(h^-1 g)^2 / eps, with h^-1 g formed by the
 * group law. */
double or_log_kernel(const double *g, const double *h, double w1, double w2, double w3, double eps, int dist)
{
    double hi[3], u[3];
    or_group_inv(h, hi);
    or_group_mul(hi, g, u);
    return -or_rho2(u[0], u[1], u[2], w1, w2, w3, dist) / eps;
}

/* Tabulated log-kernel (the Gibbs kernel of Sec. 4.2 on the grid):
 * lk[((o*nth + i)*D + (dy+r))*D + (dx+r)], D = 2r+1, is log K(h^-1 g)
 * for an output voxel g = (dx/nx, dy/ny, theta_o) and an input voxel h = (0, 0, theta_i).
 * By left invariance only the spatial offset g - h and the two orientations matter. */
void or_taps(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
             double *lk)
{
    int D = 2 * r + 1;
    for (int o = 0; o < nth; ++o)
        for (int i = 0; i < nth; ++i)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    double g[3] = {(double)dx / nx, (double)dy / ny, 2.0 * OR_PI * o / nth};
                    double h[3] = {0.0, 0.0, 2.0 * OR_PI * i / nth};
                    lk[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] =
                        or_log_kernel(g, h, w1, w2, w3, eps, dist);
                }
}

/* Input voxel index for output (y, x) and offset (dy, dx), or -1 when it lies outside a
 * zero-boundary grid. */
static long or_src(int y, int x, int dy, int dx, int nx, int ny, int periodic)
{
    int sy = y - dy, sx = x - dx;
    if (periodic) {
        sy = ((sy % ny) + ny) % ny;
        sx = ((sx % nx) + nx) % nx;
    } else if (sy < 0 || sy >= ny || sx < 0 || sx >= nx) {
        return -1;
    }
    return (long)sy * nx + sx;
}

/* The group convolution of Sec. 4.2, (K * f)(g) = sum_h K(h^-1 g) f(h) with unit Haar weights:
 * out[b][y][x][o] = sum_{i, dy, dx} K_o,i(dx, dy) f[b][y-dy][x-dx][i]. */
void or_conv_lin(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                 int periodic, int batch, const double *f, double *out)
{
    int D = 2 * r + 1;
    size_t V = (size_t)nx * ny * nth;
    size_t ntap = (size_t)nth * nth * D * D;
    double *kt = (double *)malloc(sizeof(double) * ntap);
    or_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, kt);
    for (size_t t = 0; t < ntap; ++t) kt[t] = exp(kt[t]);
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < batch; ++b)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int o = 0; o < nth; ++o) {
                    double acc = 0.0;
                    for (int i = 0; i < nth; ++i)
                        for (int dy = -r; dy <= r; ++dy)
                            for (int dx = -r; dx <= r; ++dx) {
                                long s = or_src(y, x, dy, dx, nx, ny, periodic);
                                if (s < 0) continue;
                                acc += kt[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] *
                                       f[b * V + (size_t)s * nth + i];
                            }
                    out[b * V + ((size_t)y * nx + x) * nth + o] = acc;
                }
    free(kt);
}

/* One output of the log-domain convolution: log sum_{i, dy, dx} exp(lk + lf[b][y-dy][x-dx][i])
 * evaluated as M + log(sum exp(term - M)) with M the largest term.  A term below M - 746 has
 * exp(term - M) == +0.0 in double precision, so skipping its exp() leaves the sum bit-identical.
 * Entries of lf equal to -inf are zero densities and contribute no term. */
static double or_conv_log_one(int nx, int ny, int nth, int r, const double *lk, int periodic,
                              const double *lf_b, int y, int x, int o)
{
    int D = 2 * r + 1;
    double M = -INFINITY;
    for (int i = 0; i < nth; ++i)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                long s = or_src(y, x, dy, dx, nx, ny, periodic);
                if (s < 0) continue;
                double t = lk[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] + lf_b[(size_t)s * nth + i];
                if (t > M) M = t;
            }
    double acc = 0.0;
    if (M > -INFINITY) {
        for (int i = 0; i < nth; ++i)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    long s = or_src(y, x, dy, dx, nx, ny, periodic);
                    if (s < 0) continue;
                    double t = lk[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] +
                               lf_b[(size_t)s * nth + i] - M;
                    if (t < -746.0) continue;
                    acc += exp(t);
                }
    }
    return M + log(acc);
}

/* lout = log(K * exp(lf)) for every output (Sec. 4.2 in the log domain). */
void or_conv_log(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                 int periodic, int batch, const double *lf, double *lout)
{
    int D = 2 * r + 1;
    size_t V = (size_t)nx * ny * nth;
    double *lk = (double *)malloc(sizeof(double) * (size_t)nth * nth * D * D);
    or_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, lk);
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < batch; ++b)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int o = 0; o < nth; ++o)
                    lout[b * V + ((size_t)y * nx + x) * nth + o] =
                        or_conv_log_one(nx, ny, nth, r, lk, periodic, lf + b * V, y, x, o);
    free(lk);
}

/* The same as or_conv_log at the npts outputs whose flat indices (layout [b][y][x][o]) are idx[k]:
 * lout[k] = log(K * exp(lf))(idx[k]).  For grids too large to convolve whole on the CPU. */
void or_conv_log_points(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                        int periodic, const double *lf, long npts, const long *idx, double *lout)
{
    int D = 2 * r + 1;
    size_t V = (size_t)nx * ny * nth;
    double *lk = (double *)malloc(sizeof(double) * (size_t)nth * nth * D * D);
    or_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, lk);
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < npts; ++k) {
        long f = idx[k];
        long b = f / (long)V, g = f % (long)V;
        int o = (int)(g % nth);
        long p = g / nth;
        int x = (int)(p % nx), y = (int)(p / nx);
        lout[k] = or_conv_log_one(nx, ny, nth, r, lk, periodic, lf + b * V, y, x, o);
    }
    free(lk);
}

/* Marginal violation and mass after an iteration (the paper gives no stopping rule; these
 * are the quantities a stopping rule would use): mass = sum mu,
 * viol = sum_i lambda_i ||d_i - mu||_1 / ||mu||_1. */
static void or_stats_lin(size_t V, int n, const double *lam, const double *d, const double *mu,
                         double *stats)
{
    double mass = 0.0, viol = 0.0;
    for (size_t g = 0; g < V; ++g) mass += mu[g];
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (size_t g = 0; g < V; ++g) s += fabs(d[(size_t)i * V + g] - mu[g]);
        viol += lam[i] * s;
    }
    stats[0] = mass;
    stats[1] = viol / mass;
}

/* Appendix A, literally: v_i = w_i = 1; for j = 1..iters: mu = 1; for each i:
 * w_i = mu_i / (K v_i), d_i = v_i (K w_i), mu *= d_i^lambda_i; then v_i *= mu / d_i.
 * Returns mu of the last iteration.  Optional outputs (NULL to skip): v, w, d as [n][V]
 * arrays and stats = {mass, viol}. */
void or_barycenter_lin(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                       int periodic, int n, const double *mu_in, const double *lam, int iters,
                       double *bary, double *v_out, double *w_out, double *d_out, double *stats)
{
    size_t V = (size_t)nx * ny * nth;
    double *v = (double *)malloc(sizeof(double) * V * n);
    double *w = (double *)malloc(sizeof(double) * V * n);
    double *d = (double *)malloc(sizeof(double) * V * n);
    double *kv = (double *)malloc(sizeof(double) * V);
    double *mu = (double *)malloc(sizeof(double) * V);
    for (size_t g = 0; g < V * n; ++g) { v[g] = 1.0; w[g] = 1.0; d[g] = 0.0; }
    for (size_t g = 0; g < V; ++g) mu[g] = 1.0;
    for (int j = 0; j < iters; ++j) {
        for (size_t g = 0; g < V; ++g) mu[g] = 1.0;
        for (int i = 0; i < n; ++i) {
            double *vi = v + (size_t)i * V, *wi = w + (size_t)i * V, *di = d + (size_t)i * V;
            or_conv_lin(nx, ny, nth, r, w1, w2, w3, eps, dist, periodic, 1, vi, kv);
            for (size_t g = 0; g < V; ++g) wi[g] = mu_in[(size_t)i * V + g] / kv[g];
            or_conv_lin(nx, ny, nth, r, w1, w2, w3, eps, dist, periodic, 1, wi, kv);
            for (size_t g = 0; g < V; ++g) di[g] = vi[g] * kv[g];
            if (lam[i] != 0.0)
                for (size_t g = 0; g < V; ++g) mu[g] *= pow(di[g], lam[i]);
        }
        for (int i = 0; i < n; ++i)
            for (size_t g = 0; g < V; ++g)
                v[(size_t)i * V + g] = v[(size_t)i * V + g] * mu[g] / d[(size_t)i * V + g];
    }
    memcpy(bary, mu, sizeof(double) * V);
    if (v_out) memcpy(v_out, v, sizeof(double) * V * n);
    if (w_out) memcpy(w_out, w, sizeof(double) * V * n);
    if (d_out) memcpy(d_out, d, sizeof(double) * V * n);
    if (stats) or_stats_lin(V, n, lam, d, mu, stats);
    free(v); free(w); free(d); free(kv); free(mu);
}

/* Appendix A with each scaling vector held as its natural logarithm:
 * lv_i = lw_i = 0; for j = 1..iters: L = 0; for each i:
 * lw_i = log mu_i - log(K v_i), ld_i = lv_i + log(K w_i), L += lambda_i ld_i;
 * then lv_i += L - ld_i.  Returns exp(L) of the last iteration.  Optional outputs as in
 * or_barycenter_lin but as logarithms (lv, lw, ld), plus the final L. */
void or_barycenter_log(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                       int periodic, int n, const double *mu_in, const double *lam, int iters,
                       double *bary, double *lv_out, double *lw_out, double *ld_out, double *L_out,
                       double *stats)
{
    size_t V = (size_t)nx * ny * nth;
    double *lmu = (double *)malloc(sizeof(double) * V * n);
    double *lv = (double *)malloc(sizeof(double) * V * n);
    double *lw = (double *)malloc(sizeof(double) * V * n);
    double *ld = (double *)malloc(sizeof(double) * V * n);
    double *lkv = (double *)malloc(sizeof(double) * V);
    double *L = (double *)malloc(sizeof(double) * V);
    for (size_t g = 0; g < V * n; ++g) {
        lmu[g] = log(mu_in[g]);
        lv[g] = 0.0; lw[g] = 0.0; ld[g] = 0.0;
    }
    for (size_t g = 0; g < V; ++g) L[g] = 0.0;
    for (int j = 0; j < iters; ++j) {
        for (size_t g = 0; g < V; ++g) L[g] = 0.0;
        for (int i = 0; i < n; ++i) {
            double *lvi = lv + (size_t)i * V, *lwi = lw + (size_t)i * V, *ldi = ld + (size_t)i * V;
            or_conv_log(nx, ny, nth, r, w1, w2, w3, eps, dist, periodic, 1, lvi, lkv);
            for (size_t g = 0; g < V; ++g) lwi[g] = lmu[(size_t)i * V + g] - lkv[g];
            or_conv_log(nx, ny, nth, r, w1, w2, w3, eps, dist, periodic, 1, lwi, lkv);
            for (size_t g = 0; g < V; ++g) ldi[g] = lvi[g] + lkv[g];
            if (lam[i] != 0.0)
                for (size_t g = 0; g < V; ++g) L[g] += lam[i] * ldi[g];
        }
        for (int i = 0; i < n; ++i)
            for (size_t g = 0; g < V; ++g)
                lv[(size_t)i * V + g] += L[g] - ld[(size_t)i * V + g];
    }
    for (size_t g = 0; g < V; ++g) bary[g] = exp(L[g]);
    if (lv_out) memcpy(lv_out, lv, sizeof(double) * V * n);
    if (lw_out) memcpy(lw_out, lw, sizeof(double) * V * n);
    if (ld_out) memcpy(ld_out, ld, sizeof(double) * V * n);
    if (L_out) memcpy(L_out, L, sizeof(double) * V);
    if (stats) {
        double *d = (double *)malloc(sizeof(double) * V * n);
        for (size_t g = 0; g < V * n; ++g) d[g] = exp(ld[g]);
        or_stats_lin(V, n, lam, d, bary, stats);
        free(d);
    }
    free(lmu); free(lv); free(lw); free(ld); free(lkv); free(L);
}

/* Cost-weighted tap table for the plan's cost <c, pi> of Sec. 4.1:
 * lkc = log(c(h^-1 g) K(h^-1 g)) = log(rho_b^2) - rho_b^2 / eps in the
 * layout of or_taps; -inf where the cost vanishes (the identity tap). */
void or_cost_taps(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                  double *lkc)
{
    int D = 2 * r + 1;
    for (int o = 0; o < nth; ++o)
        for (int i = 0; i < nth; ++i)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    double g[3] = {(double)dx / nx, (double)dy / ny, 2.0 * OR_PI * o / nth};
                    double h[3] = {0.0, 0.0, 2.0 * OR_PI * i / nth};
                    double hi[3], u[3];
                    or_group_inv(h, hi);
                    or_group_mul(hi, g, u);
                    double c = or_rho2(u[0], u[1], u[2], w1, w2, w3, dist);
                    lkc[((size_t)(o * nth + i) * D + (dy + r)) * D + (dx + r)] =
                        (c > 0.0 ? log(c) : -INFINITY) - c / eps;
                }
}

/* lout = log(sum_h T(h^-1 g) exp(lf(h))) for a tabulated log-kernel T (layout of or_taps). */
static void or_conv_log_table(int nx, int ny, int nth, int r, const double *lk, int periodic,
                              const double *lf, double *lout)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int o = 0; o < nth; ++o)
                lout[((size_t)y * nx + x) * nth + o] = or_conv_log_one(nx, ny, nth, r, lk, periodic, lf, y, x, o);
}

/* Entropic transport between mu and nu (Sec. 4.1).  The scaling iterations with both marginals
 * prescribed, started from b = 1, `iters` times:
 *   log a = log mu - log(K b),   log b = log nu - log(K a)
 * (K symmetric, so K^T = K).  Then, for the plan pi(g, h) = a(g) K(h^-1 g) b(h):
 *   res[0] = <c, pi> = sum_g a(g) (cK * b)(g)          transport cost, c = rho_b^2
 *   res[1] = eps (<mu, log a> + <nu, log b>)            dual objective (entries with mu or nu = 0 skipped)
 *   res[2] = sum pi = sum_g a(g) (K * b)(g)             plan mass
 *   res[3] = ||a (K * b) - mu||_1 / ||mu||_1            first-marginal violation (the second
 *                                                       holds exactly after the b-step)
 * la_out / lb_out (may be NULL) receive log a and log b. */
void or_w2_log(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
               int periodic, const double *mu, const double *nu, int iters, double *res,
               double *la_out, double *lb_out)
{
    int D = 2 * r + 1;
    size_t V = (size_t)nx * ny * nth, ntap = (size_t)nth * nth * D * D;
    double *lk = (double *)malloc(sizeof(double) * ntap);
    double *lkc = (double *)malloc(sizeof(double) * ntap);
    or_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, lk);
    or_cost_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, lkc);
    double *la = (double *)malloc(sizeof(double) * V);
    double *lb = (double *)malloc(sizeof(double) * V);
    double *t = (double *)malloc(sizeof(double) * V);
    for (size_t g = 0; g < V; ++g) {
        la[g] = 0.0;
        lb[g] = 0.0;
    }
    for (int j = 0; j < iters; ++j) {
        or_conv_log_table(nx, ny, nth, r, lk, periodic, lb, t);
        for (size_t g = 0; g < V; ++g) la[g] = log(mu[g]) - t[g];
        or_conv_log_table(nx, ny, nth, r, lk, periodic, la, t);
        for (size_t g = 0; g < V; ++g) lb[g] = log(nu[g]) - t[g];
    }
    double mass = 0.0, dev = 0.0, msum = 0.0, cost = 0.0, dual = 0.0;
    or_conv_log_table(nx, ny, nth, r, lk, periodic, lb, t);
    for (size_t g = 0; g < V; ++g) {
        double m = exp(la[g] + t[g]);
        mass += m;
        dev += fabs(m - mu[g]);
        msum += mu[g];
    }
    or_conv_log_table(nx, ny, nth, r, lkc, periodic, lb, t);
    for (size_t g = 0; g < V; ++g) {
        cost += exp(la[g] + t[g]);
        if (mu[g] > 0.0) dual += mu[g] * la[g];
        if (nu[g] > 0.0) dual += nu[g] * lb[g];
    }
    res[0] = cost;
    res[1] = eps * dual;
    res[2] = mass;
    res[3] = dev / msum;
    if (la_out) memcpy(la_out, la, sizeof(double) * V);
    if (lb_out) memcpy(lb_out, lb, sizeof(double) * V);
    free(lk); free(lkc); free(la); free(lb); free(t);
}

/* The JKO step's KL-proximal map (Sec. 2.2 Eq. (GF_JKO), Sec. 6.4, which only cites it; derived here):
 * prox of sigma F, F(s) = s^m / (m - 1) per voxel (unit Haar weight), at z = exp(lz):
 * prox(z) = argmin_s sigma s^m / (m - 1) + s log(s / z) - s.  Setting the derivative to zero,
 * u = log s solves u + c exp((m - 1) u) = lz with c = sigma m / (m - 1); the left side is increasing
 * and convex in u, so Newton's method converges from any start (from the right monotonically).
 * Returns u = log prox(z); lz = -inf gives -inf. */
double or_prox_log(double lz, double sigma, double m)
{
    if (lz == -INFINITY) return -INFINITY;
    double c = sigma * m / (m - 1.0), q = m - 1.0;
    double u = lz;
    /* a start no worse than lz when c exp(q lz) is large: the root has c exp(q u) <= |lz| + 1 */
    double alt = log((fabs(lz) + 1.0) / c) / q;
    if (alt < u) u = alt;
    for (int it = 0; it < 200; ++it) {
        double e = c * exp(q * u);
        double f = u + e - lz, fp = 1.0 + q * e;
        double step = f / fp;
        u -= step;
        if (fabs(step) <= 1e-15 * (1.0 + fabs(u))) break;
    }
    return u;
}

/* `steps` entropic JKO steps mu_{k+1} = argmin_nu W_eps(mu_k, nu) + tau F(nu) from mu_0 (Sec. 2.2
 * Eq. (GF_JKO) with the entropic scheme of Sec. 4.1).  Each step runs `iters` scaling iterations
 * from b = 1:
 *   log a = log mu_k - log(K b)                       (prox of the constraint on the 1st marginal)
 *   u = log prox_{(tau/eps) F}(K a),  log b = u - log(K a)     (prox of tau F on the 2nd marginal)
 * and mu_{k+1} = exp(u) of the last iteration (= b (K a), the plan's second marginal).
 * mu_out: V values; stats[0] = sum mu_out, stats[1] = ||a (K b) - mu_k||_1 / ||mu_k||_1 of the last
 * step (its first-marginal violation). */
void or_jko_log(int nx, int ny, int nth, int r, double w1, double w2, double w3, double eps, int dist,
                int periodic, const double *mu0, double tau, double m, int steps, int iters, double *mu_out,
                double *stats)
{
    int D = 2 * r + 1;
    size_t V = (size_t)nx * ny * nth;
    double *lk = (double *)malloc(sizeof(double) * (size_t)nth * nth * D * D);
    or_taps(nx, ny, nth, r, w1, w2, w3, eps, dist, lk);
    double *lmu = (double *)malloc(sizeof(double) * V);
    double *la = (double *)malloc(sizeof(double) * V);
    double *lb = (double *)malloc(sizeof(double) * V);
    double *t = (double *)malloc(sizeof(double) * V);
    double *u = (double *)malloc(sizeof(double) * V);
    double sigma = tau / eps, viol = 0.0;
    for (size_t g = 0; g < V; ++g) lmu[g] = log(mu0[g]);
    for (int k = 0; k < steps; ++k) {
        for (size_t g = 0; g < V; ++g) lb[g] = 0.0;
        for (int j = 0; j < iters; ++j) {
            or_conv_log_table(nx, ny, nth, r, lk, periodic, lb, t);
            for (size_t g = 0; g < V; ++g) la[g] = lmu[g] - t[g];
            or_conv_log_table(nx, ny, nth, r, lk, periodic, la, t);
            for (size_t g = 0; g < V; ++g) {
                u[g] = or_prox_log(t[g], sigma, m);
                lb[g] = u[g] - t[g];
            }
        }
        /* first-marginal violation of this step */
        or_conv_log_table(nx, ny, nth, r, lk, periodic, lb, t);
        double dev = 0.0, msum = 0.0;
        for (size_t g = 0; g < V; ++g) {
            double mk = exp(lmu[g]);
            dev += fabs(exp(la[g] + t[g]) - mk);
            msum += mk;
        }
        viol = dev / msum;
        for (size_t g = 0; g < V; ++g) lmu[g] = u[g];
    }
    double mass = 0.0;
    for (size_t g = 0; g < V; ++g) {
        mu_out[g] = exp(lmu[g]);
        mass += mu_out[g];
    }
    stats[0] = mass;
    stats[1] = viol;
    free(lk); free(lmu); free(la); free(lb); free(t); free(u);
}
