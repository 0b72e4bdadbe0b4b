/*
 * Plain FP64 reference ("oracle") for the boundary-element hot path of
 * "Monte Carlo Rendering to Diffusion Curves with Differential BEM".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the tests, the smoke check and the bench's CPU-baseline leg load it.
 * It shares no source with the CUDA library.
 *
 * What it computes, per (point x, straight panel a->b):
 *
 *   G_eps(x,z)      = -(1/4pi) log(|z-x|^2 + eps^2)        regularised Eq. (fundsol), Sec. 3.1.3
 *   dG_eps/dn_z     = -(1/2pi) n.(z-x) / (|z-x|^2 + eps^2)  only the denominator is regularised
 *   S(x)  = int_panel G_eps dz          (single layer, weight of w_c in Eq. (handleterm))
 *   Dl(x) = int_panel dG_eps/dn_z dz    (double layer, weight of w_d in Eq. (handleterm))
 *
 * with n the right normal of a->b.  Both integrals are taken exactly (closed
 * forms in the panel's frame: t = (z-x).tau, h = (a-x).n, h'^2 = h^2+eps^2):
 *
 *   Phi = atan(t2/h') - atan(t1/h') = atan2(h' L, h'^2 + t1 t2)
 *   S   = -(1/4pi) [ t2 log q2 - t1 log q1 - 2 L + 2 h' Phi ],  qi = ti^2 + h'^2
 *   Dl  = -(1/2pi) (h/h') Phi
 *
 * Derivatives with respect to the endpoints a, b follow Sec. 3.2.2: the
 * panel is written in parametric form z(s) = a + s (b-a), s in [0,1], so the
 * integration domain no longer moves, and the integrands are differentiated
 * under the integral; the resulting 1-D integrals of rational functions of t
 * are again closed forms (I_k = int t^k/q, J_k = int t^k/q^2).
 *
 * The boundary of the image is unregularised: the double-layer integral of
 * segment j seen from x is -phi_j(x)/(2pi), phi_j the signed angle that the
 * segment subtends at x (Eq. (bie), (fundsol)).
 *
 * Points are processed independently (OpenMP over points); every output
 * element is written by exactly one thread, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---- one panel, one point ------------------------------------------------ */

typedef struct {
    double L, tx, ty, nx, ny;     /* length, unit tangent, right normal */
    double dax, day, dbx, dby;    /* a - x, b - x */
    double t1, t2, h;
} frame_t;

static int make_frame(const double *ab, double x, double y, frame_t *f)
{
    double ex = ab[2] - ab[0], ey = ab[3] - ab[1];
    f->L = sqrt(ex * ex + ey * ey);
    if (!(f->L > 0.0)) return 0;
    f->tx = ex / f->L;  f->ty = ey / f->L;
    f->nx = f->ty;      f->ny = -f->tx;
    f->dax = ab[0] - x; f->day = ab[1] - y;
    f->dbx = ab[2] - x; f->dby = ab[3] - y;
    f->t1 = f->dax * f->tx + f->day * f->ty;
    f->t2 = f->dbx * f->tx + f->dby * f->ty;
    f->h  = f->dax * f->nx + f->day * f->ny;
    return 1;
}

/* Single layer S and (optionally) dS/da, dS/db. */
static void single_layer(const frame_t *f, double eps, double *S, double *dSa, double *dSb)
{
    double hp2 = f->h * f->h + eps * eps, hp = sqrt(hp2);
    double t1 = f->t1, t2 = f->t2, L = f->L;
    double q1 = t1 * t1 + hp2, q2 = t2 * t2 + hp2;
    double L1 = log(q1), L2 = log(q2);
    double Phi = atan2(hp * L, hp2 + t1 * t2);
    /* t log(t^2 + h'^2) -> 0 as t -> 0 when h' = 0 (eps = 0 at an endpoint) */
    double T1 = (t1 != 0.0) ? t1 * L1 : 0.0, T2 = (t2 != 0.0) ? t2 * L2 : 0.0;
    double Lam = T2 - T1 - 2.0 * L + 2.0 * hp * Phi;
    *S = -Lam / (4.0 * ORC_PI);
    if (!dSa) return;
    /* I0 = int dt/q = Phi/h',  I1 = int t/q,  I2 = int t^2/q */
    double hI0 = (hp > 0.0) ? f->h * Phi / hp : 0.0;       /* h * I0 */
    double I0 = (hp > 0.0) ? Phi / hp : 0.0;
    double I1 = 0.5 * (L2 - L1);
    double I2 = L - hp * Phi;
    /* dS/da = -(1/4pi)[ -tau Lam/L + (2/L)(tau (t2 I1 - I2) + h n (t2 I0 - I1)) ] */
    double ta = -Lam / L + (2.0 / L) * (t2 * I1 - I2);
    double na = (2.0 / L) * (t2 * hI0 - f->h * I1);
    double tb = Lam / L + (2.0 / L) * (I2 - t1 * I1);
    double nb = (2.0 / L) * (f->h * I1 - t1 * hI0);
    (void)I0;
    dSa[0] = -(ta * f->tx + na * f->nx) / (4.0 * ORC_PI);
    dSa[1] = -(ta * f->ty + na * f->ny) / (4.0 * ORC_PI);
    dSb[0] = -(tb * f->tx + nb * f->nx) / (4.0 * ORC_PI);
    dSb[1] = -(tb * f->ty + nb * f->ny) / (4.0 * ORC_PI);
}

/* Double layer Dl and (optionally) dDl/da, dDl/db. */
static void double_layer(const frame_t *f, double eps, double *Dl, double *dDa, double *dDb)
{
    double hp2 = f->h * f->h + eps * eps, hp = sqrt(hp2);
    double t1 = f->t1, t2 = f->t2, L = f->L;
    double Phi = atan2(hp * L, hp2 + t1 * t2);
    /* c = (a-x) x (b-x) = h L;  Dl = -(1/2pi) c int_0^1 ds/q(s) = -(1/2pi) c I0 / L */
    double c = f->dax * f->dby - f->day * f->dbx;
    double I0 = (hp > 0.0) ? Phi / hp : 0.0;
    *Dl = -(c * I0 / L) / (2.0 * ORC_PI);
    if (!dDa) return;
    double q1 = t1 * t1 + hp2, q2 = t2 * t2 + hp2;
    double J0 = (t2 / q2 - t1 / q1) / (2.0 * hp2) + Phi / (2.0 * hp2 * hp);
    double J1 = 0.5 * (1.0 / q1 - 1.0 / q2);
    double J2 = I0 - hp2 * J0;
    double s = -2.0 / (L * L);
    /* d/da int_0^1 ds/q = -(2/L^2)[tau (t2 J1 - J2) + h n (t2 J0 - J1)] */
    double ta = s * (t2 * J1 - J2), na = s * f->h * (t2 * J0 - J1);
    double tb = s * (J2 - t1 * J1), nb = s * f->h * (J1 - t1 * J0);
    double dIa0 = ta * f->tx + na * f->nx, dIa1 = ta * f->ty + na * f->ny;
    double dIb0 = tb * f->tx + nb * f->nx, dIb1 = tb * f->ty + nb * f->ny;
    /* dc/da = (dby, -dbx),  dc/db = (-day, dax) */
    double k = I0 / L;
    dDa[0] = -( f->dby * k + c * dIa0) / (2.0 * ORC_PI);
    dDa[1] = -(-f->dbx * k + c * dIa1) / (2.0 * ORC_PI);
    dDb[0] = -(-f->day * k + c * dIb0) / (2.0 * ORC_PI);
    dDb[1] = -( f->dax * k + c * dIb1) / (2.0 * ORC_PI);
}

/* ---- exported kernels ------------------------------------------------------ */

/*
 * Per-pair values (and derivatives) for n points x P panels.
 *   xy[n][2], ab[P][4] = (ax, ay, bx, by)
 *   S[n][P], Dl[n][P]                    (always)
 *   dS[n][P][4], dDl[n][P][4] = d/d(ax, ay, bx, by)   (if non-NULL)
 * S uses eps_c (the w_c term), Dl uses eps_d (the w_d term).
 */
void orc_pair_terms(int64_t n, const double *xy, int64_t P, const double *ab,
                    double eps_d, double eps_c,
                    double *S, double *Dl, double *dS, double *dDl)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        for (int64_t p = 0; p < P; ++p) {
            frame_t f;
            int64_t o = i * P + p;
            if (!make_frame(ab + 4 * p, xy[2 * i], xy[2 * i + 1], &f)) {
                S[o] = 0.0; Dl[o] = 0.0;
                if (dS) for (int k = 0; k < 4; ++k) { dS[4 * o + k] = 0.0; dDl[4 * o + k] = 0.0; }
                continue;
            }
            if (dS) {
                single_layer(&f, eps_c, &S[o], &dS[4 * o], &dS[4 * o + 2]);
                double_layer(&f, eps_d, &Dl[o], &dDl[4 * o], &dDl[4 * o + 2]);
            } else {
                single_layer(&f, eps_c, &S[o], NULL, NULL);
                double_layer(&f, eps_d, &Dl[o], NULL, NULL);
            }
        }
    }
}

/*
 * Handle term of Eq. (handleterm) summed over panels with constant jumps:
 *   f_c(x) = sum_p [ -wd[p][c] Dl_p(x) + wc[p][c] S_p(x) ],   out[n][3]
 */
void orc_handle_field(int64_t n, const double *xy, int64_t P, const double *ab,
                      const double *wd, const double *wc, double eps_d, double eps_c,
                      double *out)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t p = 0; p < P; ++p) {
            frame_t f;
            double S, Dl;
            if (!make_frame(ab + 4 * p, xy[2 * i], xy[2 * i + 1], &f)) continue;
            single_layer(&f, eps_c, &S, NULL, NULL);
            double_layer(&f, eps_d, &Dl, NULL, NULL);
            for (int c = 0; c < 3; ++c)
                acc[c] += -wd[3 * p + c] * Dl + wc[3 * p + c] * S;
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] = acc[c];
    }
}

/*
 * Signed angle phi_j(x) subtended by boundary segment j (a_j -> b_j) at x:
 *   phi = atan2((a-x) x (b-x), (a-x).(b-x)),   out[n][m]
 * The boundary double-layer integral of segment j is -phi_j/(2 pi).
 */
void orc_angles(int64_t n, const double *xy, int64_t m, const double *seg, double *out)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        for (int64_t j = 0; j < m; ++j) {
            double ax = seg[4 * j] - x, ay = seg[4 * j + 1] - y;
            double bx = seg[4 * j + 2] - x, by = seg[4 * j + 3] - y;
            out[i * m + j] = atan2(ax * by - ay * bx, ax * bx + ay * by);
        }
    }
}

/*
 * Boundary term of the interior representation (Eq. (bie) with alpha = 1):
 *   out_c(x) = sum_j phi_j(x)/(2 pi) * ub[j][c],   out[n][3]
 */
void orc_boundary_field(int64_t n, const double *xy, int64_t m, const double *seg,
                        const double *ub, double *out)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < m; ++j) {
            double ax = seg[4 * j] - x, ay = seg[4 * j + 1] - y;
            double bx = seg[4 * j + 2] - x, by = seg[4 * j + 3] - y;
            double phi = atan2(ax * by - ay * bx, ax * bx + ay * by) / (2.0 * ORC_PI);
            for (int c = 0; c < 3; ++c) acc[c] += phi * ub[3 * j + c];
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] = acc[c];
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
