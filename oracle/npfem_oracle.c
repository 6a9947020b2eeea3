/*
 * npFEM oracle: a plain, slow FP64 CPU restatement of one npFEM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path in paper_1903_06479_gb300/csrc.
 *
 * Method: Kotsalos, Latt & Chopard, "Bridging the computational gap between
 * mesoscopic and continuum modeling of red blood cells for fully resolved blood
 * flow", arXiv:1903.06479.  Every function below names the section / equation it
 * follows.  Where the paper is silent, the choice made is stated in place and
 * marked "reading" in the comments.  The code favours the literal form over speed:
 * dense n x n matrices, a dense Cholesky factor of the constant Hessian
 * approximation (never its inverse), an explicit 2x2 eigen-solve for the principal
 * stretches, and root bracketing plus bisection for the SL(2) projection.
 *
 * Layout: positions, velocities, forces and gradients are AoS doubles [n][3].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* material vector order (all physical units in um, us, pN) */
enum { M_B = 0, M_C, M_D, M_KBEND, M_KVOL, M_KMAT, M_RHO, M_ALPHA, M_BETA, M_KAPPA, M_COUNT };

typedef struct or_model {
    int n, nt;
    int *tri;        /* [nt][3] */
    double *X;       /* rest positions [n][3] */
    double *Dm_inv;  /* [nt][2][2], row-major */
    double *W;       /* rest triangle areas [nt] */
    /* one-ring neighbour lists with cotangent weights c_ij (already divided by
       twice the mixed Voronoi area of i) */
    int *ring_ptr, *ring_idx;
    double *ring_c;
    double *Avor;    /* mixed Voronoi area per vertex */
    double *dg;      /* rest Laplacian vector delta_g per vertex [n][3] */
    double *Nrest;   /* rest area-weighted vertex normal [n][3] */
    double *mass;    /* lumped mass per vertex [n] */
    double *L;       /* dense n x n, sum_i w_i G_i^T G_i */
    double *Mt;      /* dense n x n, M~ = M + h (alpha M + beta L) */
    double *Hc;      /* Cholesky factor (lower) of H~ = M~/h^2 + L */
    double *Mc;      /* Cholesky factor (lower) of M~ */
    double V0, A0, lbar, mtotal, h;
    double mat[M_COUNT];
} or_model;

typedef struct or_opts {
    int lbfgs_m;       /* history window; 0 = plain preconditioned descent */
    int max_iter;      /* cap on quasi-Newton iterations */
    double tol;        /* residual tolerance */
    double c1, c2;     /* Armijo and curvature constants */
    int max_halvings;  /* line-search trials after alpha = 1 */
    int fixed_alpha;   /* 1 = take alpha = 1 without a line search (local/global) */
} or_opts;

typedef struct or_stats {
    int iterations, evaluations, status, pad;
    double residual, objective, volume, area;
} or_stats;

enum { OR_OK = 0, OR_MAXITER = 1, OR_LINESEARCH_FAIL = 2, OR_NONFINITE = 3 };

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static void v3sub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double v3dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v3cross(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double v3norm(const double *a) { return sqrt(v3dot(a, a)); }

/* ------------------------------------------------------------------------ */
/* dense Cholesky (lower) and solve                                          */
/* ------------------------------------------------------------------------ */
static int cholesky(double *A, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / d;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0.0;
    }
    return 0;
}

/* solve (C C^T) z = b in place for one column with stride 3 (AoS component c) */
static void chol_solve_comp(const double *Cf, int n, double *b, int c)
{
    for (int i = 0; i < n; ++i) {
        double s = b[3 * i + c];
        for (int k = 0; k < i; ++k) s -= Cf[(size_t)i * n + k] * b[3 * k + c];
        b[3 * i + c] = s / Cf[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[3 * i + c];
        for (int k = i + 1; k < n; ++k) s -= Cf[(size_t)k * n + i] * b[3 * k + c];
        b[3 * i + c] = s / Cf[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------------------ */
/* SL(2) projection of the principal stretches (Sec. 2.1.2, area preservation). */
/* Reading: Sigma* = diag(a, 1/a) minimising (a - s1)^2 + (1/a - s2)^2; its      */
/* stationary points are the positive roots of f(a) = a^4 - s1 a^3 + s2 a - 1.  */
/* All positive roots are bracketed on the monotone pieces of f and bisected;   */
/* the one with the smallest distance wins, ties going to a >= 1.               */
/* ------------------------------------------------------------------------ */
static double quart(double a, double s1, double s2) { return ((a - s1) * a * a) * a + s2 * a - 1.0; }
static double quart_d(double a, double s1, double s2) { return 4.0 * a * a * a - 3.0 * s1 * a * a + s2; }

static double bisect(double (*f)(double, double, double), double lo, double hi, double s1, double s2)
{
    double flo = f(lo, s1, s2);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = f(mid, s1, s2);
        if (fm == 0.0) return mid;
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double or_sl2_project(double s1, double s2)
{
    /* f'' = 12 a^2 - 6 s1 a vanishes at a = s1/2, so f' is monotone on (0, s1/2] and
       on [s1/2, inf); f'(0) = s2 >= 0.  Collect the critical points of f. */
    double hi = s1 + 2.0; /* f(s1 + 1) >= 0, so all roots are below s1 + 2 */
    double knots[6];
    int nk = 0;
    knots[nk++] = 0.0;
    double m = 0.5 * s1;
    if (m > 0.0) {
        if ((quart_d(0.0, s1, s2) > 0) != (quart_d(m, s1, s2) > 0)) knots[nk++] = bisect(quart_d, 0.0, m, s1, s2);
        knots[nk++] = m;
        if ((quart_d(m, s1, s2) > 0) != (quart_d(hi, s1, s2) > 0)) knots[nk++] = bisect(quart_d, m, hi, s1, s2);
    }
    knots[nk++] = hi;
    double best = 1.0, bestphi = INFINITY;
    for (int k = 0; k + 1 < nk; ++k) {
        double lo = knots[k], up = knots[k + 1];
        if (!(up > lo)) continue;
        double flo = quart(lo, s1, s2), fup = quart(up, s1, s2);
        double r;
        if (flo == 0.0 && lo > 0.0) r = lo;
        else if ((flo < 0) != (fup < 0) || fup == 0.0) r = (fup == 0.0) ? up : bisect(quart, lo, up, s1, s2);
        else continue;
        if (!(r > 0.0)) continue;
        double phi = (r - s1) * (r - s1) + (1.0 / r - s2) * (1.0 / r - s2);
        if (phi < bestphi || (phi == bestphi && r >= 1.0)) { bestphi = phi; best = r; }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* thin SVD of a 3x2 deformation gradient through the 2x2 eigenproblem of F^T F */
/* (Sec. 2.1.3: P(F) = U P(Sigma) V^T).  Returns -1 for a degenerate element.   */
/* ------------------------------------------------------------------------ */
static int svd32(const double F[3][2], double U[3][2], double sig[2], double V[2][2])
{
    double a = F[0][0] * F[0][0] + F[1][0] * F[1][0] + F[2][0] * F[2][0];
    double b = F[0][0] * F[0][1] + F[1][0] * F[1][1] + F[2][0] * F[2][1];
    double c = F[0][1] * F[0][1] + F[1][1] * F[1][1] + F[2][1] * F[2][1];
    double mean = 0.5 * (a + c), dif = 0.5 * (a - c);
    double rad = sqrt(dif * dif + b * b);
    double mu1 = mean + rad, mu2 = mean - rad;
    double v1x, v1y;
    if (rad == 0.0) { v1x = 1.0; v1y = 0.0; }
    else if (dif >= 0.0) { v1x = dif + rad; v1y = b; }
    else { v1x = b; v1y = rad - dif; }
    double nv = sqrt(v1x * v1x + v1y * v1y);
    v1x /= nv; v1y /= nv;
    V[0][0] = v1x; V[1][0] = v1y;   /* first column */
    V[0][1] = -v1y; V[1][1] = v1x;  /* second column */
    if (mu2 < 0.0) mu2 = 0.0;
    sig[0] = sqrt(mu1);
    sig[1] = sqrt(mu2);
    if (!(sig[1] > 0.0) || !isfinite(sig[0])) return -1;
    for (int k = 0; k < 2; ++k)
        for (int r = 0; r < 3; ++r) U[r][k] = (F[r][0] * V[0][k] + F[r][1] * V[1][k]) / sig[k];
    return 0;
}

/* F = D_s D_m^{-1} for triangle t (Appendix B; D_s = [x_j - x_i, x_k - x_i]) */
static void deformation_gradient(const or_model *m, const double *x, int t, double F[3][2])
{
    const int *tv = m->tri + 3 * t;
    double e1[3], e2[3];
    v3sub(x + 3 * tv[1], x + 3 * tv[0], e1);
    v3sub(x + 3 * tv[2], x + 3 * tv[0], e2);
    const double *Di = m->Dm_inv + 4 * t;
    for (int r = 0; r < 3; ++r) {
        F[r][0] = e1[r] * Di[0] + e2[r] * Di[2];
        F[r][1] = e1[r] * Di[1] + e2[r] * Di[3];
    }
}

/* scatter dE/dF (3x2) to the three vertices: dE/dD_s = dE/dF D_m^{-T} */
static void scatter_dF(const or_model *m, int t, const double G[3][2], double *grad)
{
    const int *tv = m->tri + 3 * t;
    const double *Di = m->Dm_inv + 4 * t;
    for (int r = 0; r < 3; ++r) {
        double gj = G[r][0] * Di[0] + G[r][1] * Di[1];
        double gk = G[r][0] * Di[2] + G[r][1] * Di[3];
        grad[3 * tv[1] + r] += gj;
        grad[3 * tv[2] + r] += gk;
        grad[3 * tv[0] + r] -= gj + gk;
    }
}

/* ------------------------------------------------------------------------ */
/* Local area preservation, Sec. 2.1.2: E_i = (C/2) W_i ||F - T||_F^2 with      */
/* T = U Sigma* V^T, det(Sigma*) = 1; PD gradient C W_i (F - T) D_m^{-T}.       */
/* Reading: weight w_i = C * rest area (the constant-L requirement).            */
/* ------------------------------------------------------------------------ */
double or_energy_area(const or_model *m, const double *x, double *grad, int *bad)
{
    double E = 0.0, k = m->mat[M_C];
    for (int t = 0; t < m->nt; ++t) {
        double F[3][2], U[3][2], s[2], V[2][2];
        deformation_gradient(m, x, t, F);
        if (svd32(F, U, s, V)) { if (bad) *bad = 1; continue; }
        double a = or_sl2_project(s[0], s[1]);
        double ss[2] = {a, 1.0 / a};
        double T[3][2], D[3][2], n2 = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 2; ++cc) {
                T[r][cc] = U[r][0] * ss[0] * V[cc][0] + U[r][1] * ss[1] * V[cc][1];
                D[r][cc] = F[r][cc] - T[r][cc];
                n2 += D[r][cc] * D[r][cc];
            }
        E += 0.5 * k * m->W[t] * n2;
        if (grad) {
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 2; ++cc) D[r][cc] *= k * m->W[t];
            scatter_dF(m, t, D, grad);
        }
    }
    return E;
}

/* Modified Skalak strain energy, Sec. 2.1.3: f(l) = B l^4/8 - B l^2/4 + D (l-1)^4/4,
   reading: shifted by +B/8 so that f(1) = 0; the area part g is dropped.
   E_i = W_i (f(l1) + f(l2)); dE/dF = W_i U diag(f'(l1), f'(l2)) V^T. */
double or_skalak_f(double l, double B, double D)
{
    double q = (l - 1.0) * (l - 1.0);
    return B * l * l * l * l / 8.0 - B * l * l / 4.0 + D * q * q / 4.0 + B / 8.0;
}
double or_skalak_fp(double l, double B, double D)
{
    return B * l * l * l / 2.0 - B * l / 2.0 + D * (l - 1.0) * (l - 1.0) * (l - 1.0);
}

double or_energy_skalak(const or_model *m, const double *x, double *grad, int *bad)
{
    double E = 0.0, B = m->mat[M_B], Dd = m->mat[M_D];
    for (int t = 0; t < m->nt; ++t) {
        double F[3][2], U[3][2], s[2], V[2][2];
        deformation_gradient(m, x, t, F);
        if (svd32(F, U, s, V)) { if (bad) *bad = 1; continue; }
        E += m->W[t] * (or_skalak_f(s[0], B, Dd) + or_skalak_f(s[1], B, Dd));
        if (grad) {
            double p0 = or_skalak_fp(s[0], B, Dd) * m->W[t], p1 = or_skalak_fp(s[1], B, Dd) * m->W[t];
            double G[3][2];
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 2; ++cc) G[r][cc] = U[r][0] * p0 * V[cc][0] + U[r][1] * p1 * V[cc][1];
            scatter_dF(m, t, G, grad);
        }
    }
    return E;
}

/* ------------------------------------------------------------------------ */
/* Bending, Sec. 2.1.2 (Eq. BendingDiscretizedPotential): per vertex i          */
/* E_i = (k/2) A_i || X_f c - R X_g c ||^2, R in SO(3).  The closest rotated     */
/* rest vector is p = |delta_g| delta_f / |delta_f|; PD gradient k A_i G_i^T     */
/* (delta_f - p) with G_i x = sum_j c_ij (x_j - x_i).                           */
/* ------------------------------------------------------------------------ */
static void area_weighted_normals(const or_model *m, const double *x, double *N)
{
    memset(N, 0, sizeof(double) * 3 * m->n);
    for (int t = 0; t < m->nt; ++t) {
        const int *tv = m->tri + 3 * t;
        double e1[3], e2[3], c[3];
        v3sub(x + 3 * tv[1], x + 3 * tv[0], e1);
        v3sub(x + 3 * tv[2], x + 3 * tv[0], e2);
        v3cross(e1, e2, c); /* = 2 A n */
        for (int a = 0; a < 3; ++a)
            for (int r = 0; r < 3; ++r) N[3 * tv[a] + r] += 0.5 * c[r];
    }
}

double or_energy_bend(const or_model *m, const double *x, double *grad)
{
    double E = 0.0, k = m->mat[M_KBEND];
    double *Ncur = NULL;
    for (int i = 0; i < m->n; ++i) {
        double df[3] = {0, 0, 0}, csum = 0.0;
        for (int q = m->ring_ptr[i]; q < m->ring_ptr[i + 1]; ++q) {
            int j = m->ring_idx[q];
            double c = m->ring_c[q];
            for (int r = 0; r < 3; ++r) df[r] += c * (x[3 * j + r] - x[3 * i + r]);
            csum += c;
        }
        double ng = v3norm(m->dg + 3 * i), nf = v3norm(df);
        double p[3] = {0, 0, 0};
        if (ng > 0.0) {
            if (nf > 1e-12 * ng) {
                for (int r = 0; r < 3; ++r) p[r] = ng * df[r] / nf;
            } else {
                /* reading: delta_f ~ 0 leaves the rotation free; use the current
                   vertex normal, oriented as delta_g is to the rest normal */
                if (!Ncur) { Ncur = (double *)malloc(sizeof(double) * 3 * m->n); area_weighted_normals(m, x, Ncur); }
                double nn = v3norm(Ncur + 3 * i);
                double sgn = v3dot(m->dg + 3 * i, m->Nrest + 3 * i) >= 0.0 ? 1.0 : -1.0;
                if (nn > 0.0)
                    for (int r = 0; r < 3; ++r) p[r] = sgn * ng * Ncur[3 * i + r] / nn;
            }
        }
        double rr[3] = {df[0] - p[0], df[1] - p[1], df[2] - p[2]};
        double w = k * m->Avor[i];
        E += 0.5 * w * v3dot(rr, rr);
        if (grad) {
            for (int q = m->ring_ptr[i]; q < m->ring_ptr[i + 1]; ++q) {
                int j = m->ring_idx[q];
                double c = m->ring_c[q];
                for (int r = 0; r < 3; ++r) grad[3 * j + r] += w * c * rr[r];
            }
            for (int r = 0; r < 3; ++r) grad[3 * i + r] -= w * csum * rr[r];
        }
    }
    free(Ncur);
    return E;
}

/* ------------------------------------------------------------------------ */
/* Global volume conservation, Sec. 2.1.2: V = (1/9) sum_i A_i (x1+x2+x3)^T n_i, */
/* C = V - V0, grad C_k = (1/3) sum of area-weighted normals of the triangles    */
/* around k, projection dx = -C grad C / |grad C|^2.                            */
/* E = (w/2)|p - x|^2 = (w/2) C^2/|grad C|^2; PD gradient w (x - p).           */
/* ------------------------------------------------------------------------ */
double or_volume(const or_model *m, const double *x)
{
    double V = 0.0;
    for (int t = 0; t < m->nt; ++t) {
        const int *tv = m->tri + 3 * t;
        double e1[3], e2[3], An[3], s[3];
        v3sub(x + 3 * tv[1], x + 3 * tv[0], e1);
        v3sub(x + 3 * tv[2], x + 3 * tv[0], e2);
        v3cross(e1, e2, An);
        for (int r = 0; r < 3; ++r) { An[r] *= 0.5; s[r] = x[3 * tv[0] + r] + x[3 * tv[1] + r] + x[3 * tv[2] + r]; }
        V += v3dot(An, s) / 9.0;
    }
    return V;
}

double or_area(const or_model *m, const double *x)
{
    double A = 0.0;
    for (int t = 0; t < m->nt; ++t) {
        const int *tv = m->tri + 3 * t;
        double e1[3], e2[3], c[3];
        v3sub(x + 3 * tv[1], x + 3 * tv[0], e1);
        v3sub(x + 3 * tv[2], x + 3 * tv[0], e2);
        v3cross(e1, e2, c);
        A += 0.5 * v3norm(c);
    }
    return A;
}

/* gradC [n][3] = (1/3) sum A_j n_j over incident triangles */
void or_volume_gradient(const or_model *m, const double *x, double *gradC)
{
    area_weighted_normals(m, x, gradC);
    for (int i = 0; i < 3 * m->n; ++i) gradC[i] /= 3.0;
}

double or_energy_vol(const or_model *m, const double *x, double *grad, double *vol_out)
{
    double V = or_volume(m, x);
    if (vol_out) *vol_out = V;
    double *gc = (double *)malloc(sizeof(double) * 3 * m->n);
    or_volume_gradient(m, x, gc);
    double g2 = 0.0;
    for (int i = 0; i < 3 * m->n; ++i) g2 += gc[i] * gc[i];
    double C = V - m->V0, w = m->mat[M_KVOL];
    double E = 0.5 * w * C * C / g2;
    if (grad)
        for (int i = 0; i < 3 * m->n; ++i) grad[i] += w * (C / g2) * gc[i];
    free(gc);
    return E;
}

/* ------------------------------------------------------------------------ */
/* Objective (Eq. GeneralizedObjectiveFunction) and gradient                   */
/* (Eq. GeneralizedObjectiveFunctionDerivative):                               */
/* g = (1/2h^2) tr((x-y)^T M~ (x-y)) + PD energies + non-PD energies.           */
/* parts (optional, 6): inertia, area, skalak, bend, volume-energy, V.          */
/* ------------------------------------------------------------------------ */
/* Collision energy of Sec. 3.3 (non-PD part of Eq. GeneralizedObjectiveFunction):  */
/* vertex i with a plane (unit normal n_i, offset c_i; n_i = 0: none) penetrates    */
/* the neighbouring body while d_i = c_i - n_i . x_i > 0; its desired position p_i   */
/* is x_i moved onto the plane, so E = (w/2) |p_i - x_i|^2 = (w/2) d_i^2 and the force */
/* w (p_i - x_i) = w d_i n_i.  The test d_i > 0 is made at every evaluation, which   */
/* cancels the term as soon as the vertex no longer penetrates.                       */
double or_energy_collision(const or_model *m, const double *x, const double *col, double wcol, double *grad)
{
    double E = 0.0;
    if (!col) return 0.0;
    for (int i = 0; i < m->n; ++i) {
        const double *pl = col + 4 * i;
        if (pl[0] == 0.0 && pl[1] == 0.0 && pl[2] == 0.0) continue;
        double d = pl[3] - v3dot(pl, x + 3 * i);
        if (!(d > 0.0)) continue;
        E += 0.5 * wcol * d * d;
        if (grad)
            for (int r = 0; r < 3; ++r) grad[3 * i + r] -= wcol * d * pl[r];
    }
    return E;
}

static double objective_col(const or_model *m, const double *x, const double *y, double *grad, double *parts, int *bad,
                            const double *col, double wcol);

double or_objective(const or_model *m, const double *x, const double *y, double *grad, double *parts, int *bad)
{
    return objective_col(m, x, y, grad, parts, bad, NULL, 0.0);
}

double or_objective_col(const or_model *m, const double *x, const double *y, double *grad, double *parts, int *bad,
                        const double *col, double wcol)
{
    return objective_col(m, x, y, grad, parts, bad, col, wcol);
}

static double objective_col(const or_model *m, const double *x, const double *y, double *grad, double *parts, int *bad,
                            const double *col, double wcol)
{
    int n = m->n;
    double h2 = m->h * m->h;
    if (grad) memset(grad, 0, sizeof(double) * 3 * n);
    double Ein = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < n; ++i) {
            double mi = 0.0;
            for (int j = 0; j < n; ++j) mi += m->Mt[(size_t)i * n + j] * (x[3 * j + c] - y[3 * j + c]);
            Ein += 0.5 / h2 * (x[3 * i + c] - y[3 * i + c]) * mi;
            if (grad) grad[3 * i + c] += mi / h2;
        }
    double Ea = or_energy_area(m, x, grad, bad);
    double Es = or_energy_skalak(m, x, grad, bad);
    double Eb = or_energy_bend(m, x, grad);
    double V = 0.0;
    double Ev = or_energy_vol(m, x, grad, &V);
    double Ec = or_energy_collision(m, x, col, wcol, grad);
    if (parts) { parts[0] = Ein; parts[1] = Ea; parts[2] = Es; parts[3] = Eb; parts[4] = Ev; parts[5] = V; }
    return Ein + Ea + Es + Eb + Ev + Ec;
}

/* internal energy only (no inertia), gradient overwritten */
double or_internal_energy(const or_model *m, const double *x, double *grad)
{
    if (grad) memset(grad, 0, sizeof(double) * 3 * m->n);
    int bad = 0;
    double E = or_energy_area(m, x, grad, &bad) + or_energy_skalak(m, x, grad, &bad) + or_energy_bend(m, x, grad);
    E += or_energy_vol(m, x, grad, NULL);
    return E;
}

/* ------------------------------------------------------------------------ */
/* rest-state precompute and operator assembly (Sec. 2.1.1, 2.1.2, 2.1.4)      */
/* ------------------------------------------------------------------------ */
static double corner_cot(const double *a, const double *b, const double *c)
{
    /* cotangent of the angle at a in triangle (a, b, c) */
    double u[3], v[3], w[3];
    v3sub(b, a, u);
    v3sub(c, a, v);
    v3cross(u, v, w);
    return v3dot(u, v) / v3norm(w);
}

void or_destroy(or_model *m)
{
    if (!m) return;
    free(m->tri); free(m->X); free(m->Dm_inv); free(m->W); free(m->ring_ptr); free(m->ring_idx);
    free(m->ring_c); free(m->Avor); free(m->dg); free(m->Nrest); free(m->mass); free(m->L); free(m->Mt);
    free(m->Hc); free(m->Mc);
    free(m);
}

/* Validates a closed, consistently oriented 2-manifold: every directed edge (a,b)
   occurs exactly once and its reverse (b,a) exactly once. */
static int check_mesh(int n, int nt, const int *tri)
{
    if (n < 4 || nt < 4) return -1;
    char *dir = (char *)calloc((size_t)n * n, 1);
    if (!dir) return -1;
    int ok = 0;
    for (int t = 0; t < nt && !ok; ++t)
        for (int a = 0; a < 3; ++a) {
            int i = tri[3 * t + a], j = tri[3 * t + (a + 1) % 3];
            if (i < 0 || i >= n || j < 0 || j >= n || i == j) { ok = -1; break; }
            if (dir[(size_t)i * n + j]) { ok = -1; break; }
            dir[(size_t)i * n + j] = 1;
        }
    for (size_t i = 0; i < (size_t)n && !ok; ++i)
        for (size_t j = 0; j < (size_t)n; ++j)
            if (dir[i * n + j] != dir[j * n + i]) { ok = -1; break; }
    free(dir);
    return ok;
}

or_model *or_create(int n, int nt, const int *tri, const double *rest, const double *mat, double dt, int equal_mass)
{
    if (check_mesh(n, nt, tri)) return NULL;
    or_model *m = (or_model *)calloc(1, sizeof(or_model));
    m->n = n; m->nt = nt; m->h = dt;
    memcpy(m->mat, mat, sizeof(double) * M_COUNT);
    m->tri = (int *)malloc(sizeof(int) * 3 * nt);
    memcpy(m->tri, tri, sizeof(int) * 3 * nt);
    m->X = (double *)malloc(sizeof(double) * 3 * n);
    memcpy(m->X, rest, sizeof(double) * 3 * n);
    m->Dm_inv = (double *)malloc(sizeof(double) * 4 * nt);
    m->W = (double *)malloc(sizeof(double) * nt);
    m->Avor = (double *)calloc(n, sizeof(double));
    m->dg = (double *)calloc(3 * n, sizeof(double));
    m->Nrest = (double *)calloc(3 * n, sizeof(double));
    m->mass = (double *)calloc(n, sizeof(double));
    double *cotw = (double *)calloc((size_t)n * n, sizeof(double)); /* sum of cotangents per edge */
    char *adj = (char *)calloc((size_t)n * n, 1);
    double *bary = (double *)calloc(n, sizeof(double));

    /* D_m in a 2D frame of the rest triangle (Appendix B), rest areas W, angles */
    double Atot = 0.0, lsum = 0.0;
    int ecount = 0;
    for (int t = 0; t < nt; ++t) {
        const int *tv = tri + 3 * t;
        const double *Xi = rest + 3 * tv[0], *Xj = rest + 3 * tv[1], *Xk = rest + 3 * tv[2];
        double E1[3], E2[3], nrm[3], b1[3], b2[3];
        v3sub(Xj, Xi, E1);
        v3sub(Xk, Xi, E2);
        v3cross(E1, E2, nrm);
        double l1 = v3norm(E1);
        for (int r = 0; r < 3; ++r) b1[r] = E1[r] / l1;
        v3cross(nrm, b1, b2);
        double nb2 = v3norm(b2);
        for (int r = 0; r < 3; ++r) b2[r] /= nb2;
        double Dm[2][2] = {{v3dot(E1, b1), v3dot(E2, b1)}, {v3dot(E1, b2), v3dot(E2, b2)}};
        double det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
        m->Dm_inv[4 * t + 0] = Dm[1][1] / det;
        m->Dm_inv[4 * t + 1] = -Dm[0][1] / det;
        m->Dm_inv[4 * t + 2] = -Dm[1][0] / det;
        m->Dm_inv[4 * t + 3] = Dm[0][0] / det;
        double T = 0.5 * v3norm(nrm);
        m->W[t] = T;
        Atot += T;
        for (int a = 0; a < 3; ++a) {
            bary[tv[a]] += T / 3.0;
            for (int r = 0; r < 3; ++r) m->Nrest[3 * tv[a] + r] += 0.5 * nrm[r];
        }
        /* cotangent weights: the angle at corner a is opposite edge (a+1, a+2) */
        const double *P[3] = {Xi, Xj, Xk};
        double ct[3];
        for (int a = 0; a < 3; ++a) {
            ct[a] = corner_cot(P[a], P[(a + 1) % 3], P[(a + 2) % 3]);
            int p = tv[(a + 1) % 3], q = tv[(a + 2) % 3];
            cotw[(size_t)p * n + q] += ct[a];
            cotw[(size_t)q * n + p] += ct[a];
            if (!adj[(size_t)p * n + q]) { lsum += sqrt(pow(P[(a + 1) % 3][0] - P[(a + 2) % 3][0], 2) + pow(P[(a + 1) % 3][1] - P[(a + 2) % 3][1], 2) + pow(P[(a + 1) % 3][2] - P[(a + 2) % 3][2], 2)); ecount++; }
            adj[(size_t)p * n + q] = adj[(size_t)q * n + p] = 1;
        }
        /* mixed Voronoi area (Meyer et al. 2003): Voronoi share for non-obtuse
           triangles, T/2 to the obtuse corner and T/4 to the others otherwise */
        int obtuse = -1;
        for (int a = 0; a < 3; ++a) if (ct[a] < 0.0) obtuse = a;
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, c = (a + 2) % 3;
            if (obtuse < 0) {
                double lab[3], lac[3];
                v3sub(P[b], P[a], lab);
                v3sub(P[c], P[a], lac);
                m->Avor[tv[a]] += (v3dot(lab, lab) * ct[c] + v3dot(lac, lac) * ct[b]) / 8.0;
            } else {
                m->Avor[tv[a]] += (a == obtuse) ? T / 2.0 : T / 4.0;
            }
        }
    }
    m->A0 = Atot;
    m->lbar = lsum / ecount;

    /* one-ring lists with c_ij = (cot a + cot b) / (2 A_i) (reading of "cotangent
       weights divided by the Voronoi area") */
    m->ring_ptr = (int *)calloc(n + 1, sizeof(int));
    int nnz = 0;
    for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) if (adj[(size_t)i * n + j]) nnz++;
    m->ring_idx = (int *)malloc(sizeof(int) * nnz);
    m->ring_c = (double *)malloc(sizeof(double) * nnz);
    nnz = 0;
    for (int i = 0; i < n; ++i) {
        m->ring_ptr[i] = nnz;
        for (int j = 0; j < n; ++j)
            if (adj[(size_t)i * n + j]) {
                m->ring_idx[nnz] = j;
                m->ring_c[nnz] = cotw[(size_t)i * n + j] / (2.0 * m->Avor[i]);
                nnz++;
            }
    }
    m->ring_ptr[n] = nnz;
    for (int i = 0; i < n; ++i)
        for (int q = m->ring_ptr[i]; q < m->ring_ptr[i + 1]; ++q)
            for (int r = 0; r < 3; ++r) m->dg[3 * i + r] += m->ring_c[q] * (rest[3 * m->ring_idx[q] + r] - rest[3 * i + r]);

    m->V0 = or_volume(m, rest);
    /* lumped mass (Sec. 2.1.1): total mass rho V0 spread by barycentric area
       share (reading) or equally */
    m->mtotal = mat[M_RHO] * m->V0;
    for (int i = 0; i < n; ++i) m->mass[i] = equal_mass ? m->mtotal / n : m->mtotal * bary[i] / Atot;

    /* L = sum_i w_i G_i^T G_i (Eq. fullyDeveloped_g), n x n */
    m->L = (double *)calloc((size_t)n * n, sizeof(double));
    double kA = mat[M_C] + mat[M_KMAT];
    for (int t = 0; t < nt; ++t) {
        const int *tv = tri + 3 * t;
        const double *Di = m->Dm_inv + 4 * t;
        for (int a = 0; a < 2; ++a) {
            double g[3] = {-(Di[0 * 2 + a] + Di[1 * 2 + a]), Di[0 * 2 + a], Di[1 * 2 + a]};
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) m->L[(size_t)tv[p] * n + tv[q]] += kA * m->W[t] * g[p] * g[q];
        }
    }
    for (int i = 0; i < n; ++i) {
        double w = mat[M_KBEND] * m->Avor[i];
        int deg = m->ring_ptr[i + 1] - m->ring_ptr[i];
        int *idx = (int *)malloc(sizeof(int) * (deg + 1));
        double *g = (double *)malloc(sizeof(double) * (deg + 1));
        double cs = 0.0;
        for (int q = 0; q < deg; ++q) { idx[q] = m->ring_idx[m->ring_ptr[i] + q]; g[q] = m->ring_c[m->ring_ptr[i] + q]; cs += g[q]; }
        idx[deg] = i; g[deg] = -cs;
        for (int p = 0; p <= deg; ++p)
            for (int q = 0; q <= deg; ++q) m->L[(size_t)idx[p] * n + idx[q]] += w * g[p] * g[q];
        free(idx); free(g);
        m->L[(size_t)i * n + i] += mat[M_KVOL]; /* volume: G = I, w = k_vol */
    }

    /* Rayleigh damping C = alpha M + beta L (Sec. 2.1.4, L standing in for K);
       M~ = M + h C; H~ = M~/h^2 + L (Sec. 2.1.1) */
    m->Mt = (double *)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            m->Mt[(size_t)i * n + j] = (i == j ? m->mass[i] * (1.0 + dt * mat[M_ALPHA]) : 0.0) + dt * mat[M_BETA] * m->L[(size_t)i * n + j];
    m->Hc = (double *)malloc(sizeof(double) * n * n);
    m->Mc = (double *)malloc(sizeof(double) * n * n);
    for (size_t i = 0; i < (size_t)n * n; ++i) { m->Hc[i] = m->Mt[i] / (dt * dt) + m->L[i]; m->Mc[i] = m->Mt[i]; }
    int bad = cholesky(m->Hc, n) || cholesky(m->Mc, n);
    free(cotw); free(adj); free(bary);
    if (bad) { or_destroy(m); return NULL; }
    return m;
}

/* ------------------------------------------------------------------------ */
/* queries used by the tests                                                  */
/* ------------------------------------------------------------------------ */
int or_n(const or_model *m) { return m->n; }
int or_nt(const or_model *m) { return m->nt; }
void or_rest_info(const or_model *m, double *out)
{
    out[0] = m->V0; out[1] = m->A0; out[2] = m->lbar; out[3] = m->mtotal;
}
void or_masses(const or_model *m, double *o) { memcpy(o, m->mass, sizeof(double) * m->n); }
void or_voronoi(const or_model *m, double *o) { memcpy(o, m->Avor, sizeof(double) * m->n); }
void or_laplacian(const or_model *m, double *o) { memcpy(o, m->L, sizeof(double) * m->n * m->n); }
void or_hessian(const or_model *m, double *o)
{
    size_t n = m->n;
    for (size_t i = 0; i < n * n; ++i) o[i] = m->Mt[i] / (m->h * m->h) + m->L[i];
}
/* apply H~^{-1} to an AoS vector (three columns) in place */
void or_apply_hinv(const or_model *m, double *b)
{
    for (int c = 0; c < 3; ++c) chol_solve_comp(m->Hc, m->n, b, c);
}

/* First guess, Algorithm 1: y = x_n + h M~^{-1} M v_n + h^2 M~^{-1} F_ext */
void or_first_guess(const or_model *m, const double *x, const double *v, const double *f, double *y)
{
    int n = m->n;
    double h = m->h;
    double *b = (double *)malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) b[3 * i + c] = h * m->mass[i] * v[3 * i + c] + h * h * f[3 * i + c];
    for (int c = 0; c < 3; ++c) chol_solve_comp(m->Mc, n, b, c);
    for (int i = 0; i < 3 * n; ++i) y[i] = x[i] + b[i];
    free(b);
}

/* Reading of the stopping rule: r = RMS_i(h^2 |grad_i| / m_i) / lbar0 */
double or_residual(const or_model *m, const double *grad)
{
    double s = 0.0, h2 = m->h * m->h;
    for (int i = 0; i < m->n; ++i) {
        double q = h2 * v3norm(grad + 3 * i) / m->mass[i];
        s += q * q;
    }
    return sqrt(s / m->n) / m->lbar;
}

/* ------------------------------------------------------------------------ */
/* Quasi-Newton solve of Algorithm 1 with the L-BFGS direction (Nocedal &      */
/* Wright Algorithm 7.4, initial matrix H~^{-1}) and the backtracking line      */
/* search alpha = 1, 1/2, ...  x holds x^(1) on entry and x_{n+1} on exit.     */
/* ------------------------------------------------------------------------ */
static double dot3n(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int i = 0; i < 3 * n; ++i) s += a[i] * b[i];
    return s;
}

static int solve_core(const or_model *m, double *x, const double *y, const or_opts *o, or_stats *st,
                      const double *col, double wcol, double *S_io, double *Y_io, int *count_io);

static int solve_col(const or_model *m, double *x, const double *y, const or_opts *o, or_stats *st, const double *col,
                     double wcol)
{
    return solve_core(m, x, y, o, st, col, wcol, NULL, NULL, NULL);
}

int or_solve(const or_model *m, double *x, const double *y, const or_opts *o, or_stats *st)
{
    return solve_col(m, x, y, o, st, NULL, 0.0);
}

/* The same solve starting from *count_io history pairs carried over from an earlier  */
/* solve (an addition to the paper's Algorithm 1, which starts every time step with   */
/* an empty history): S_io, Y_io hold lbfgs_m vectors of 3n (AoS) each, the oldest    */
/* pair first; on return they hold the solve's final pairs in the same order and      */
/* *count_io their number (0 after a failed line search or a non-finite state).       */
int or_solve_carry(const or_model *m, double *x, const double *y, const or_opts *o, or_stats *st, double *S_io,
                   double *Y_io, int *count_io)
{
    return solve_core(m, x, y, o, st, NULL, 0.0, S_io, Y_io, count_io);
}

static int solve_core(const or_model *m, double *x, const double *y, const or_opts *o, or_stats *st,
                      const double *col, double wcol, double *S_io, double *Y_io, int *count_io)
{
    int n = m->n, N = 3 * n, M = o->lbfgs_m;
    size_t vb = sizeof(double) * N;
    double *g = (double *)malloc(vb), *d = (double *)malloc(vb), *xt = (double *)malloc(vb), *gt = (double *)malloc(vb);
    double *S = (double *)malloc(vb * (M > 0 ? M : 1)), *Y = (double *)malloc(vb * (M > 0 ? M : 1));
    double *rho = (double *)malloc(sizeof(double) * (M > 0 ? M : 1)), *al = (double *)malloc(sizeof(double) * (M > 0 ? M : 1));
    int head = 0, count = 0, bad = 0;
    if (count_io && *count_io > 0 && M > 0) {
        /* carried pairs into slots 0..count-1, the newest last */
        count = *count_io < M ? *count_io : M;
        memcpy(S, S_io, vb * count);
        memcpy(Y, Y_io, vb * count);
        for (int i = 0; i < count; ++i) rho[i] = 1.0 / dot3n(S + (size_t)i * N, Y + (size_t)i * N, n);
        head = count % M;
    }
    st->iterations = 0; st->evaluations = 1; st->status = OR_OK;
    double parts[6];
    double E = objective_col(m, x, y, g, parts, &bad, col, wcol);
    int k = 0;
    for (;;) {
        double r = or_residual(m, g);
        st->residual = r;
        if (bad || !isfinite(E) || !isfinite(r)) { st->status = OR_NONFINITE; break; }
        if (r <= o->tol) break;
        if (k >= o->max_iter) { st->status = OR_MAXITER; break; }
        /* two-loop recursion */
        memcpy(d, g, vb);
        for (int q = 0; q < count; ++q) {
            int i = (head - 1 - q + M) % M;
            al[i] = rho[i] * dot3n(S + (size_t)i * N, d, n);
            for (int e = 0; e < N; ++e) d[e] -= al[i] * Y[(size_t)i * N + e];
        }
        or_apply_hinv(m, d);
        for (int q = count - 1; q >= 0; --q) {
            int i = (head - 1 - q + M) % M;
            double be = rho[i] * dot3n(Y + (size_t)i * N, d, n);
            for (int e = 0; e < N; ++e) d[e] += S[(size_t)i * N + e] * (al[i] - be);
        }
        for (int e = 0; e < N; ++e) d[e] = -d[e];
        double gd = dot3n(g, d, n);
        if (!(gd < 0.0)) {
            /* not a descent direction: drop the history and use -H~^{-1} grad */
            count = 0;
            for (int e = 0; e < N; ++e) d[e] = g[e];
            or_apply_hinv(m, d);
            for (int e = 0; e < N; ++e) d[e] = -d[e];
            gd = dot3n(g, d, n);
        }
        double alpha = 1.0, Et = 0.0;
        int accepted = 0;
        for (int hv = 0; hv <= o->max_halvings; ++hv) {
            for (int e = 0; e < N; ++e) xt[e] = x[e] + alpha * d[e];
            bad = 0;
            Et = objective_col(m, xt, y, gt, parts, &bad, col, wcol);
            st->evaluations++;
            if (o->fixed_alpha || (!bad && Et <= E + o->c1 * alpha * gd)) { accepted = 1; break; }
            alpha *= 0.5;
        }
        if (!accepted) { st->status = OR_LINESEARCH_FAIL; count = 0; bad = 0; break; }
        /* history pair (s, y), stored when the curvature condition holds and s^T y > 0 */
        double gtd = dot3n(gt, d, n);
        if (M > 0) {
            double *s = S + (size_t)head * N, *yy = Y + (size_t)head * N;
            double sy = 0.0, ss = 0.0, yy2 = 0.0;
            for (int e = 0; e < N; ++e) {
                double se = xt[e] - x[e], ye = gt[e] - g[e];
                sy += se * ye; ss += se * se; yy2 += ye * ye;
            }
            if (gtd >= o->c2 * gd && sy > 1e-12 * sqrt(ss * yy2)) {
                for (int e = 0; e < N; ++e) { s[e] = xt[e] - x[e]; yy[e] = gt[e] - g[e]; }
                rho[head] = 1.0 / sy;
                head = (head + 1) % M;
                if (count < M) count++;
            }
        }
        memcpy(x, xt, vb);
        memcpy(g, gt, vb);
        E = Et;
        k++;
        st->iterations = k;
    }
    st->objective = E;
    st->volume = or_volume(m, x);
    st->area = or_area(m, x);
    if (count_io) {
        /* the pairs, oldest first; none after a failure */
        if (st->status == OR_NONFINITE || st->status == OR_LINESEARCH_FAIL) count = 0;
        for (int q = 0; q < count; ++q) {
            int i = (head - count + q + M) % M;
            memcpy(S_io + (size_t)q * N, S + (size_t)i * N, vb);
            memcpy(Y_io + (size_t)q * N, Y + (size_t)i * N, vb);
        }
        *count_io = count;
    }
    free(g); free(d); free(xt); free(gt); free(S); free(Y); free(rho); free(al);
    return st->status;
}

/* Post-convergence dissipation (Sec. 2.1.4, after Mueller et al. 2007):
   damp the velocity part that the best-fit rigid motion does not explain. */
void or_post_step(const or_model *m, const double *x, double *v, double kappa)
{
    int n = m->n;
    double mt = 0.0, xcm[3] = {0, 0, 0}, vcm[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        mt += m->mass[i];
        for (int r = 0; r < 3; ++r) { xcm[r] += m->mass[i] * x[3 * i + r]; vcm[r] += m->mass[i] * v[3 * i + r]; }
    }
    for (int r = 0; r < 3; ++r) { xcm[r] /= mt; vcm[r] /= mt; }
    double Lm[3] = {0, 0, 0}, I[3][3] = {{0}};
    for (int i = 0; i < n; ++i) {
        double ri[3], mv[3], c[3];
        v3sub(x + 3 * i, xcm, ri);
        for (int r = 0; r < 3; ++r) mv[r] = m->mass[i] * v[3 * i + r];
        v3cross(ri, mv, c);
        for (int r = 0; r < 3; ++r) Lm[r] += c[r];
        /* r~ r~^T = |r|^2 I - r r^T */
        double rr = v3dot(ri, ri);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) I[a][b] += m->mass[i] * ((a == b ? rr : 0.0) - ri[a] * ri[b]);
    }
    /* omega = I^{-1} L by the adjugate */
    double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) - I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                 I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
    double inv[3][3];
    inv[0][0] = (I[1][1] * I[2][2] - I[1][2] * I[2][1]) / det;
    inv[0][1] = (I[0][2] * I[2][1] - I[0][1] * I[2][2]) / det;
    inv[0][2] = (I[0][1] * I[1][2] - I[0][2] * I[1][1]) / det;
    inv[1][0] = (I[1][2] * I[2][0] - I[1][0] * I[2][2]) / det;
    inv[1][1] = (I[0][0] * I[2][2] - I[0][2] * I[2][0]) / det;
    inv[1][2] = (I[0][2] * I[1][0] - I[0][0] * I[1][2]) / det;
    inv[2][0] = (I[1][0] * I[2][1] - I[1][1] * I[2][0]) / det;
    inv[2][1] = (I[0][1] * I[2][0] - I[0][0] * I[2][1]) / det;
    inv[2][2] = (I[0][0] * I[1][1] - I[0][1] * I[1][0]) / det;
    double w[3];
    for (int a = 0; a < 3; ++a) w[a] = inv[a][0] * Lm[0] + inv[a][1] * Lm[1] + inv[a][2] * Lm[2];
    for (int i = 0; i < n; ++i) {
        double ri[3], wr[3];
        v3sub(x + 3 * i, xcm, ri);
        v3cross(w, ri, wr);
        for (int r = 0; r < 3; ++r) {
            double dv = vcm[r] + wr[r] - v[3 * i + r];
            v[3 * i + r] += kappa * dv;
        }
    }
}

/* One time step of Algorithm 1 for one cell: first guess, quasi-Newton solve,
   v_{n+1} = (x_{n+1} - x_n)/h, post-convergence dissipation. */
int or_step_col(const or_model *m, double *x, double *v, const double *f, const or_opts *o, or_stats *st,
                const double *col, double wcol);

int or_step(const or_model *m, double *x, double *v, const double *f, const or_opts *o, or_stats *st)
{
    return or_step_col(m, x, v, f, o, st, NULL, 0.0);
}

/* The same step with collision planes (n x 4, or NULL) and weight wcol. */
int or_step_col(const or_model *m, double *x, double *v, const double *f, const or_opts *o, or_stats *st,
                const double *col, double wcol)
{
    int n = m->n;
    size_t vb = sizeof(double) * 3 * n;
    double *xn = (double *)malloc(vb), *y = (double *)malloc(vb);
    memcpy(xn, x, vb);
    or_first_guess(m, xn, v, f, y);
    memcpy(x, y, vb);
    int s = solve_col(m, x, y, o, st, col, wcol);
    if (s == OR_NONFINITE) memcpy(x, xn, vb); /* keep x_n for a failed cell */
    for (int i = 0; i < 3 * n; ++i) v[i] = (x[i] - xn[i]) / m->h;
    or_post_step(m, x, v, m->mat[M_KAPPA]);
    free(xn); free(y);
    return s;
}

/* ------------------------------------------------------------------------ */
/* batch over independent cells on a pool of threads (cells are independent:  */
/* no exchange inside a step)                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_model *m;
    double *x, *v;
    const double *f;
    const or_opts *o;
    or_stats *st;
    int c0, c1, steps;
    const double *col; /* ncells x n x 4 collision planes, or NULL */
    double wcol;
} or_job;

static void *or_worker(void *arg)
{
    or_job *j = (or_job *)arg;
    size_t N = 3 * (size_t)j->m->n;
    for (int c = j->c0; c < j->c1; ++c)
        for (int s = 0; s < j->steps; ++s)
            or_step_col(j->m, j->x + c * N, j->v + c * N, j->f + c * N, j->o, j->st + c,
                        j->col ? j->col + (size_t)c * 4 * j->m->n : NULL, j->wcol);
    return NULL;
}

int or_step_batch_col(const or_model *m, int ncells, int steps, double *x, double *v, const double *f,
                      const or_opts *o, or_stats *st, int nthreads, const double *col, double wcol);

int or_step_batch(const or_model *m, int ncells, int steps, double *x, double *v, const double *f, const or_opts *o,
                  or_stats *st, int nthreads)
{
    return or_step_batch_col(m, ncells, steps, x, v, f, o, st, nthreads, NULL, 0.0);
}

int or_step_batch_col(const or_model *m, int ncells, int steps, double *x, double *v, const double *f,
                      const or_opts *o, or_stats *st, int nthreads, const double *col, double wcol)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ncells) nthreads = ncells;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    or_job *jobs = (or_job *)malloc(sizeof(or_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (or_job){m, x, v, f, o, st, (int)((long)ncells * t / nthreads), (int)((long)ncells * (t + 1) / nthreads),
                           steps, col, wcol};
        pthread_create(&th[t], NULL, or_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}

/* ======================================================================== */
/* Learned warm start (an addition to the paper's method, not in the paper): */
/* a per-vertex MLP proposes x^(1) = y + R MLP(features) before the          */
/* quasi-Newton iteration; the iteration still runs to the same residual.    */
/* Plain FP64 reference of the features, the network and its gradient.      */
/* ======================================================================== */
#define MLP_IN 9
#define MLP_H 64
#define MLP_OUT 3
/* packed parameters: W1[64][9] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
   mu[9] sigma[9] s_out[3]  (the last three are fixed normalisation constants) */
enum {
    P_W1 = 0,
    P_B1 = P_W1 + MLP_H * MLP_IN,
    P_W2 = P_B1 + MLP_H,
    P_B2 = P_W2 + MLP_H * MLP_H,
    P_W3 = P_B2 + MLP_H,
    P_B3 = P_W3 + MLP_OUT * MLP_H,
    P_MU = P_B3 + MLP_OUT,
    P_SIG = P_MU + MLP_IN,
    P_SOUT = P_SIG + MLP_IN,
    P_COUNT = P_SOUT + MLP_OUT
};

int or_mlp_nparam(void) { return P_COUNT; }

/* round a double holding an FP32 value to the nearest BF16 (ties to even), as the
   network's weights are stored */
double or_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x; /* inf / nan */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double wq(const double *P, int i, int bf16) { return bf16 ? or_bf16(P[i]) : P[i]; }

/* forward pass for one sample; keeps the activations for the backward pass.  With
   bf16 the network is the one the GPU evaluates on BF16 tensor-core operands: the
   weights, the normalised inputs (xn) and the first hidden layer (h1q, the operand
   of the second product) are rounded to BF16; h1 keeps the unrounded tanh for the
   derivative, so the gradient passes the operand rounding straight through. */
static void mlp_fwd(const double *P, const double *xraw, int bf16, double *xn, double *h1, double *h1q, double *h2,
                    double *o)
{
    for (int i = 0; i < MLP_IN; ++i) {
        xn[i] = (xraw[i] - P[P_MU + i]) / P[P_SIG + i];
        if (bf16) xn[i] = or_bf16(xn[i]);
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = P[P_B1 + j];
        for (int i = 0; i < MLP_IN; ++i) a += wq(P, P_W1 + j * MLP_IN + i, bf16) * xn[i];
        h1[j] = tanh(a);
        h1q[j] = bf16 ? or_bf16(h1[j]) : h1[j];
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = P[P_B2 + j];
        for (int i = 0; i < MLP_H; ++i) a += wq(P, P_W2 + j * MLP_H + i, bf16) * h1q[i];
        h2[j] = tanh(a);
    }
    for (int j = 0; j < MLP_OUT; ++j) {
        double a = P[P_B3 + j];
        for (int i = 0; i < MLP_H; ++i) a += wq(P, P_W3 + j * MLP_H + i, bf16) * h2[i];
        o[j] = a;
    }
}

/* network output in physical units (rest frame): o * s_out */
void or_mlp_predict(const double *P, const double *feat, int n, double *out, int bf16)
{
    double xn[MLP_IN], h1[MLP_H], h1q[MLP_H], h2[MLP_H], o[MLP_OUT];
    for (int s = 0; s < n; ++s) {
        mlp_fwd(P, feat + MLP_IN * s, bf16, xn, h1, h1q, h2, o);
        for (int c = 0; c < MLP_OUT; ++c) out[MLP_OUT * s + c] = o[c] * P[P_SOUT + c];
    }
}

/* loss = (1/n) sum_s sum_c (o_c - t_c / s_out_c)^2 and its gradient with respect to
   W1, b1, W2, b2, W3, b3 (zero for the normalisation constants); with bf16 the
   forward pass is the BF16-operand network of mlp_fwd and the gradient is taken
   through its rounded weights and operands */
double or_mlp_loss_grad(const double *P, const double *feat, const double *target, int n, double *grad, int bf16)
{
    memset(grad, 0, sizeof(double) * P_COUNT);
    double loss = 0.0;
    double xn[MLP_IN], h1[MLP_H], h1q[MLP_H], h2[MLP_H], o[MLP_OUT], d2[MLP_H], d1[MLP_H];
    for (int s = 0; s < n; ++s) {
        mlp_fwd(P, feat + MLP_IN * s, bf16, xn, h1, h1q, h2, o);
        double dout[MLP_OUT];
        for (int c = 0; c < MLP_OUT; ++c) {
            double r = o[c] - target[MLP_OUT * s + c] / P[P_SOUT + c];
            loss += r * r;
            dout[c] = 2.0 * r / n;
        }
        for (int c = 0; c < MLP_OUT; ++c) {
            grad[P_B3 + c] += dout[c];
            for (int i = 0; i < MLP_H; ++i) grad[P_W3 + c * MLP_H + i] += dout[c] * h2[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double a = 0.0;
            for (int c = 0; c < MLP_OUT; ++c) a += dout[c] * wq(P, P_W3 + c * MLP_H + i, bf16);
            d2[i] = a * (1.0 - h2[i] * h2[i]);
        }
        for (int j = 0; j < MLP_H; ++j) {
            grad[P_B2 + j] += d2[j];
            for (int i = 0; i < MLP_H; ++i) grad[P_W2 + j * MLP_H + i] += d2[j] * h1q[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double a = 0.0;
            for (int j = 0; j < MLP_H; ++j) a += d2[j] * wq(P, P_W2 + j * MLP_H + i, bf16);
            d1[i] = a * (1.0 - h1[i] * h1[i]);
        }
        for (int j = 0; j < MLP_H; ++j) {
            grad[P_B1 + j] += d1[j];
            for (int i = 0; i < MLP_IN; ++i) grad[P_W1 + j * MLP_IN + i] += d1[j] * xn[i];
        }
    }
    return loss / n;
}

/* symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations: S = V diag(w) V^T */
static void jacobi3(double S[3][3], double w[3], double V[3][3])
{
    double A[3][3];
    memcpy(A, S, sizeof(A));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
                double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) w[i] = A[i][i];
}

/* Best-fit rotation of the rest shape onto y (mass-weighted): the orthogonal polar
   factor R = A (A^T A)^{-1/2} of A = sum_i m_i (y_i - y_cm)(X_i - X_cm)^T. */
void or_best_rotation(const or_model *m, const double *y, double *Rout, double *ycm, double *xcm)
{
    int n = m->n;
    double mt = 0.0;
    for (int r = 0; r < 3; ++r) { ycm[r] = 0.0; xcm[r] = 0.0; }
    for (int i = 0; i < n; ++i) {
        mt += m->mass[i];
        for (int r = 0; r < 3; ++r) { ycm[r] += m->mass[i] * y[3 * i + r]; xcm[r] += m->mass[i] * m->X[3 * i + r]; }
    }
    for (int r = 0; r < 3; ++r) { ycm[r] /= mt; xcm[r] /= mt; }
    double A[3][3] = {{0}};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] += m->mass[i] * (y[3 * i + a] - ycm[a]) * (m->X[3 * i + b] - xcm[b]);
    double S[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[a][b] = A[0][a] * A[0][b] + A[1][a] * A[1][b] + A[2][a] * A[2][b];
    double w[3], V[3][3], Sm[3][3];
    jacobi3(S, w, V);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += V[a][k] * V[b][k] / sqrt(w[k]);
            Sm[a][b] = s;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Rout[3 * a + b] = A[a][0] * Sm[0][b] + A[a][1] * Sm[1][b] + A[a][2] * Sm[2][b];
}

/* Per-vertex raw features at the first guess y (rest frame of the best fit):
   d_i = R^T (y_i - y_cm) - (X_i - X_cm); lap_i = sum_j c_ij (d_j - d_i);
   f_i' = R^T F_ext,i h^2 / m_i.  feat: [n][9]. */
void or_ws_features(const or_model *m, const double *y, const double *f, double *feat, double *Rout)
{
    int n = m->n;
    double ycm[3], xcm[3];
    or_best_rotation(m, y, Rout, ycm, xcm);
    const double *R = Rout;
    double *d = (double *)malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += R[3 * a + b] * (y[3 * i + a] - ycm[a]);
            d[3 * i + b] = s - (m->X[3 * i + b] - xcm[b]);
        }
    for (int i = 0; i < n; ++i) {
        double lap[3] = {0, 0, 0};
        for (int q = m->ring_ptr[i]; q < m->ring_ptr[i + 1]; ++q) {
            int j = m->ring_idx[q];
            for (int r = 0; r < 3; ++r) lap[r] += m->ring_c[q] * (d[3 * j + r] - d[3 * i + r]);
        }
        double sc = m->h * m->h / m->mass[i];
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += R[3 * a + b] * f[3 * i + a];
            feat[9 * i + b] = d[3 * i + b];
            feat[9 * i + 3 + b] = lap[b];
            feat[9 * i + 6 + b] = s * sc;
        }
    }
    free(d);
}

/* Temporal network (an addition, not in the paper): along a trajectory the first       */
/* iterate is y_n + c_{n-1} + R MLP(features), c_k = x_{k+1} - y_k the converged          */
/* correction of step k, R the best-fit rotation at y_n.  Features of vertex i (9), in    */
/* the rest frame: the trend R^T (c_{n-1} - c_{n-2}), the force change as a displacement  */
/* u = R^T h^2 (F_n - F_{n-1}) / m_i, and its cotangent Laplacian over the one-ring.       */
void or_ws_features_temporal(const or_model *m, const double *y, const double *f, const double *f_prev,
                             const double *c1, const double *c2, double *feat, double *Rout)
{
    int n = m->n;
    double ycm[3], xcm[3];
    or_best_rotation(m, y, Rout, ycm, xcm);
    const double *R = Rout;
    double *u = (double *)malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i) {
        double sc = m->h * m->h / m->mass[i];
        for (int b = 0; b < 3; ++b) {
            double su = 0.0, st = 0.0;
            for (int a = 0; a < 3; ++a) {
                su += R[3 * a + b] * (f[3 * i + a] - f_prev[3 * i + a]);
                st += R[3 * a + b] * (c1[3 * i + a] - c2[3 * i + a]);
            }
            u[3 * i + b] = su * sc;
            feat[9 * i + b] = st;
        }
    }
    for (int i = 0; i < n; ++i) {
        double lap[3] = {0, 0, 0};
        for (int q = m->ring_ptr[i]; q < m->ring_ptr[i + 1]; ++q) {
            int j = m->ring_idx[q];
            for (int r = 0; r < 3; ++r) lap[r] += m->ring_c[q] * (u[3 * j + r] - u[3 * i + r]);
        }
        for (int b = 0; b < 3; ++b) {
            feat[9 * i + 3 + b] = u[3 * i + b];
            feat[9 * i + 6 + b] = lap[b];
        }
    }
    free(u);
}

/* x1 = y + c_{n-1} + R (s_out * MLP(temporal features)). */
void or_ws_guess_temporal(const or_model *m, const double *P, const double *x, const double *v, const double *f,
                          const double *f_prev, const double *c1, const double *c2, double *x1, int bf16)
{
    int n = m->n;
    double *y = (double *)malloc(sizeof(double) * 3 * n), *feat = (double *)malloc(sizeof(double) * 9 * n);
    double *o = (double *)malloc(sizeof(double) * 3 * n), R[9];
    or_first_guess(m, x, v, f, y);
    or_ws_features_temporal(m, y, f, f_prev, c1, c2, feat, R);
    or_mlp_predict(P, feat, n, o, bf16);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            x1[3 * i + a] = y[3 * i + a] + c1[3 * i + a] + R[3 * a + 0] * o[3 * i] + R[3 * a + 1] * o[3 * i + 1] +
                            R[3 * a + 2] * o[3 * i + 2];
    free(y); free(feat); free(o);
}

/* Warm-started first guess: x1 = y + R (s_out * MLP(features)). */
void or_ws_guess(const or_model *m, const double *P, const double *x, const double *v, const double *f, double *x1,
                 int bf16)
{
    int n = m->n;
    double *y = (double *)malloc(sizeof(double) * 3 * n), *feat = (double *)malloc(sizeof(double) * 9 * n);
    double *o = (double *)malloc(sizeof(double) * 3 * n), R[9];
    or_first_guess(m, x, v, f, y);
    or_ws_features(m, y, f, feat, R);
    or_mlp_predict(P, feat, n, o, bf16);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) x1[3 * i + a] = y[3 * i + a] + R[3 * a + 0] * o[3 * i] + R[3 * a + 1] * o[3 * i + 1] + R[3 * a + 2] * o[3 * i + 2];
    free(y); free(feat); free(o);
}
