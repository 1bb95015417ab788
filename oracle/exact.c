/*
 * Test infrastructure -- plain, slow FP64 CPU oracle for the Exact particle ->
 * Voronoi mapping.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load it; the product path never does.  It shares no code with
 * the CUDA library.
 *
 * Contents
 *   M4 kernel W, dW/dh, radial cumulative G           (Section 2.4.2, cubic spline truncated at 2h)
 *   analytic integral of W over one right sub-triangle pyramid
 *   signed cone decomposition of a convex cell into face pyramids and
 *     per-edge right triangles -> w_ij = int_{V_j} W(|r - x_i|, h_i) d^3r
 *                                                     (Exact mapping, Section 1 and 2.3)
 *   independent check: adaptive Gauss-Kronrod over the sphere of directions of
 *     [G(r_out) - G(r_in)] along rays (no cone decomposition, no closed form)
 *   brute-force Voronoi cells: the box clipped by the bisector of every other
 *     generator                                       (Section 2.3, Voronoi grid on the sites)
 *   all-pairs particle-cell overlap test: dist(x_i, V_j) < 2 h_i
 *   cell densities rho_j = sum_i m_i w_ij / V_j in ascending i
 *
 * Readings (the paper cites the earlier Exact-mapping work for the formula):
 *   W(r,h) = (1/(pi h^3)) w(r/h), w(q) = 1 - 1.5q^2 + 0.75q^3 (q<1),
 *            0.25(2-q)^3 (1<=q<2), 0 beyond.
 *   A pair exists iff the closed support sphere meets the cell: dist < 2h strictly.
 *
 * Compiled with -ffp-contract=off so that products and sums round one by one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Work counting (count.cpp builds this file a second time with a counting
 * number type and defines this hook); a no-op in the oracle itself. */
#ifndef ORC_COUNT_TRIANGLE
#define ORC_COUNT_TRIANGLE()
#endif

/* ------------------------------------------------------------------------ */
/* M4 cubic spline                                                          */
/* ------------------------------------------------------------------------ */

double orc_w_shape(double q)
{
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t; }
    return 0.0;
}

double orc_dw_shape(double q)
{
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) { double t = 2.0 - q; return -0.75 * t * t; }
    return 0.0;
}

double orc_W(double r, double h) { return orc_w_shape(r / h) / (ORC_PI * h * h * h); }

/* dW/dh at fixed r: W = w(r/h)/(pi h^3)  =>  dW/dh = -(3 w + q w'(q)) / (pi h^4) */
double orc_dWdh(double r, double h)
{
    double q = r / h;
    return -(3.0 * orc_w_shape(q) + q * orc_dw_shape(q)) / (ORC_PI * h * h * h * h);
}

/* g(Q) = int_0^Q w(q) q^2 dq, so that G(R,h) = int_0^R W r^2 dr = g(R/h)/pi.
 * Pieces: Q<1: Q^3/3 - 3Q^5/10 + Q^6/8;
 *         1<=Q<2: 2Q^3/3 - 3Q^4/4 + 3Q^5/10 - Q^6/24 - 1/60;  Q>=2: 1/4. */
double orc_g(double Q)
{
    if (Q < 1.0) return Q * Q * Q / 3.0 - 0.3 * pow(Q, 5) + 0.125 * pow(Q, 6);
    if (Q < 2.0)
        return 2.0 * Q * Q * Q / 3.0 - 0.75 * pow(Q, 4) + 0.3 * pow(Q, 5) - pow(Q, 6) / 24.0
               - 1.0 / 60.0;
    return 0.25;
}

double orc_G(double R, double h) { return orc_g(R / h) / ORC_PI; }

/* K(Q) = int g(Q)/Q^2 dQ, continuous, K(0) = 0:
 *   Q<1:    Q^2/6 - 3Q^4/40 + Q^5/40
 *   1<=Q<2: Q^2/3 - Q^3/4 + 3Q^4/40 - Q^5/120 + 1/(60Q) - 1/20
 *   Q>=2:   -1/(4Q) + 7/20 */
double orc_K(double Q)
{
    if (Q < 1.0) return Q * Q / 6.0 - 3.0 * pow(Q, 4) / 40.0 + pow(Q, 5) / 40.0;
    if (Q < 2.0)
        return Q * Q / 3.0 - Q * Q * Q / 4.0 + 3.0 * pow(Q, 4) / 40.0 - pow(Q, 5) / 120.0
               + 1.0 / (60.0 * Q) - 1.0 / 20.0;
    return -1.0 / (4.0 * Q) + 7.0 / 20.0;
}

/* ------------------------------------------------------------------------ */
/* One right sub-triangle                                                    */
/*                                                                           */
/* Particle p at height d above a face plane (foot P).  F is the foot of the  */
/* perpendicular from P onto an edge line, a = |PF|; tau is the coordinate    */
/* along the edge line measured from F.  All lengths in units of h:           */
/*   D = d/h, A = a/h, B^2 = D^2 + A^2 (distance from p to the edge line),    */
/*   the point at tau is at distance Q_e = sqrt(B^2 + tau^2) from p.          */
/* The pyramid from p over the right triangle (P, F, X) with X at tau = T is  */
/*   I = int_cone W = int dOmega G(R(Omega))                                   */
/*     = (D/pi) int_0^T [K(Q_e(tau)) - K(D)] A/(A^2+tau^2) dtau               */
/* (solid-angle element d*dArea/R^3, radial part via G; in-plane angle        */
/*  phi = atan(tau/A), dphi = A dtau/(A^2+tau^2)).                             */
/* With J_n(T) = int_0^T Q_e^n A/(A^2+tau^2) dtau:                              */
/*   J_0 = atan(T/A)                                                          */
/*   D J_-1 = atan(D T / (A sqrt(B^2+T^2)))                                    */
/*   J_2 = A T + D^2 J_0                                                      */
/*   J_4 = A (A^2 T + T^3/3) + 2 D^2 A T + D^4 J_0                            */
/*   J_1 = A asinh(T/B) + D^2 J_-1                                            */
/*   J_3 = A U_1 + D^2 J_1,  U_1 = int sqrt(B^2+tau^2) = T S/2 + B^2 asinh(T/B)/2 */
/*   J_5 = A U_3 + D^2 J_3,  U_3 = int (B^2+tau^2)^(3/2) = T S^3/4 + 3 B^2 U_1/4 */
/* and on each kernel region K is a combination of Q^n, n in {-1,0,2..5}.    */
/* ------------------------------------------------------------------------ */

/* D * (antiderivative of K on region `region`) from 0 to tau */
static double dprim(int region, double A, double B, double D, double tau)
{
    double S = sqrt(B * B + tau * tau);
    double ash = asinh(tau / B);
    double J0 = atan2(tau, A);
    double DJm1 = atan2(D * tau, A * S);
    double D2 = D * D;
    double J2 = A * tau + D2 * J0;
    double J4 = A * (A * A * tau + tau * tau * tau / 3.0) + 2.0 * D2 * A * tau + D2 * D2 * J0;
    double J1 = A * ash + D * DJm1;
    double U1 = 0.5 * tau * S + 0.5 * B * B * ash;
    double J3 = A * U1 + D2 * J1;
    double U3 = 0.25 * tau * S * S * S + 0.75 * B * B * U1;
    double J5 = A * U3 + D2 * J3;
    if (region == 1) return D * (J2 / 6.0 - 3.0 * J4 / 40.0 + J5 / 40.0);
    if (region == 2)
        return D * (J2 / 3.0 - J3 / 4.0 + 3.0 * J4 / 40.0 - J5 / 120.0 - J0 / 20.0) + DJm1 / 60.0;
    return -DJm1 / 4.0 + D * (7.0 / 20.0) * J0;
}

/* Integral of W (in units where the kernel integrates to 1) over the pyramid
 * from p over the right triangle with legs A (from P to F) and |T| (from F along
 * the edge); odd in T.  D = 0 or A = 0 give a degenerate pyramid (zero). */
double orc_right_triangle(double D, double A, double T)
{
    if (D <= 0.0 || A <= 0.0 || T == 0.0) return 0.0;
    ORC_COUNT_TRIANGLE();
    double sgn = T < 0.0 ? -1.0 : 1.0;
    T = fabs(T);
    double B = sqrt(D * D + A * A);
    double t1 = B < 1.0 ? sqrt(1.0 - B * B) : 0.0;   /* Q_e = 1 at tau = t1 */
    double t2 = B < 2.0 ? sqrt(4.0 - B * B) : 0.0;   /* Q_e = 2 at tau = t2 */
    double val;
    if (T <= t1) {
        val = dprim(1, A, B, D, T);
    } else if (T <= t2) {
        val = dprim(1, A, B, D, t1) + dprim(2, A, B, D, T) - dprim(2, A, B, D, t1);
    } else {
        val = dprim(1, A, B, D, t1) + dprim(2, A, B, D, t2) - dprim(2, A, B, D, t1)
              + dprim(3, A, B, D, T) - dprim(3, A, B, D, t2);
    }
    val -= D * orc_K(D) * atan2(T, A);
    return sgn * val / ORC_PI;
}

/* ------------------------------------------------------------------------ */
/* Face pyramid and cell weight by the signed cone decomposition             */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Signed contribution of one face: sigma_f * int_{cone(p, face)} W.
 * verts: nv vertices (x,y,z) ordered counter-clockwise seen from outside, n the
 * unit outward normal.  sigma_f = sign(n.(V_0 - p)): +1 when p is on the inner
 * side of the face plane.  The face is split into triangles (P, V_k, V_k+1),
 * signed by the side of the edge line P lies on, and each triangle into the two
 * right triangles at F, the foot of P on the edge line. */
double orc_face_pyramid(const double *p, double h, int nv, const double *verts, const double *n)
{
    double rel0[3] = {verts[0] - p[0], verts[1] - p[1], verts[2] - p[2]};
    double s = dot3(n, rel0);
    if (s == 0.0) return 0.0;
    double sigma = s > 0.0 ? 1.0 : -1.0;
    double D = fabs(s) / h;
    double sum = 0.0;
    for (int k = 0; k < nv; ++k) {
        const double *a = verts + 3 * k;
        const double *b = verts + 3 * ((k + 1) % nv);
        double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double L = sqrt(dot3(e, e));
        if (L == 0.0) continue;
        double eh[3] = {e[0] / L, e[1] / L, e[2] / L};
        double m[3];
        cross3(eh, n, m);                          /* in-plane outward edge normal */
        double ra[3] = {a[0] - p[0], a[1] - p[1], a[2] - p[2]};
        double rb[3] = {b[0] - p[0], b[1] - p[1], b[2] - p[2]};
        double aa = dot3(ra, m);                   /* > 0 when P is on the inner side */
        if (aa == 0.0) continue;
        double t0 = dot3(ra, eh), t1 = dot3(rb, eh);
        double A = fabs(aa) / h;
        double sg = aa > 0.0 ? 1.0 : -1.0;
        sum += sg * (orc_right_triangle(D, A, t1 / h) - orc_right_triangle(D, A, t0 / h));
    }
    return sigma * sum;
}

/* w = int_{cell} W(|r - p|, h) d^3r for a convex cell given as faces.
 * face_vert_off[f]..face_vert_off[f+1] index verts (3 doubles each). */
double orc_cell_weight(const double *p, double h, int nface, const int64_t *face_vert_off,
                       const double *verts, const double *normals)
{
    double w = 0.0;
    for (int f = 0; f < nface; ++f) {
        int64_t v0 = face_vert_off[f], v1 = face_vert_off[f + 1];
        w += orc_face_pyramid(p, h, (int)(v1 - v0), verts + 3 * v0, normals + 3 * f);
    }
    return w;
}

/* ------------------------------------------------------------------------ */
/* Independent check: integrate over directions.  For a convex cell given by   */
/* its face planes n_f.x <= c_f, the ray p + r u meets it in [r_in, r_out] and */
/*   w = int_{S^2} [G(min(r_out,2h)) - G(min(r_in,2h))] dOmega.                 */
/* Nested adaptive Gauss-Kronrod (7/15) in mu = cos(theta) and phi.           */
/* ------------------------------------------------------------------------ */

static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef double (*orc_fn)(double x, void *ctx);

static double gk15(orc_fn f, void *ctx, double a, double b, double *err)
{
    double c = 0.5 * (a + b), hl = 0.5 * (b - a);
    double fc = f(c, ctx);
    double rk = fc * gk_wk[7], rg = fc * gk_wg[3];
    for (int j = 0; j < 7; ++j) {
        double dx = hl * gk_x[j];
        double f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
        rk += gk_wk[j] * (f1 + f2);
        if (j % 2 == 1) rg += gk_wg[j / 2] * (f1 + f2);
    }
    *err = fabs((rk - rg) * hl);
    return rk * hl;
}

/* Adaptive bisection; every interval is split at least down to depth
 * min_depth so that a cell seen under a small solid angle is not missed by
 * the first 15 nodes. */
static double adapt(orc_fn f, void *ctx, double a, double b, double tol, int depth, int min_depth)
{
    double err;
    double r = gk15(f, ctx, a, b, &err);
    if (depth >= min_depth && (err <= tol || depth >= 40)) return r;
    double c = 0.5 * (a + b);
    return adapt(f, ctx, a, c, 0.5 * tol, depth + 1, min_depth)
           + adapt(f, ctx, c, b, 0.5 * tol, depth + 1, min_depth);
}

typedef struct {
    const double *p;
    double h;
    int nface;
    const double *normals;
    const double *offsets;
    double mu;
    double tol;
} ray_ctx;

static double ray_integrand(double phi, void *vctx)
{
    ray_ctx *c = (ray_ctx *)vctx;
    double st = sqrt(fmax(0.0, 1.0 - c->mu * c->mu));
    double u[3] = {st * cos(phi), st * sin(phi), c->mu};
    double rin = 0.0, rout = INFINITY;
    for (int f = 0; f < c->nface; ++f) {
        const double *n = c->normals + 3 * f;
        double den = dot3(n, u);
        double num = c->offsets[f] - dot3(n, c->p);
        if (den > 0.0) { double t = num / den; if (t < rout) rout = t; }
        else if (den < 0.0) { double t = num / den; if (t > rin) rin = t; }
        else if (num < 0.0) return 0.0;
    }
    if (!(rin < rout)) return 0.0;
    double R2 = 2.0 * c->h;
    return orc_G(fmin(rout, R2), c->h) - orc_G(fmin(rin, R2), c->h);
}

static double ray_mu(double mu, void *vctx)
{
    ray_ctx *c = (ray_ctx *)vctx;
    ray_ctx d = *c;
    d.mu = mu;
    return adapt(ray_integrand, &d, 0.0, 2.0 * ORC_PI, c->tol, 0, 5);
}

/* Quadrature of the same weight, from the face planes alone (offsets c_f). */
double orc_cell_weight_quadrature(const double *p, double h, int nface, const double *normals,
                                  const double *offsets, double tol)
{
    ray_ctx c = {p, h, nface, normals, offsets, 0.0, tol};
    return adapt(ray_mu, &c, -1.0, 1.0, tol, 0, 5);
}

/* ------------------------------------------------------------------------ */
/* Brute-force Voronoi cell: the box clipped by the bisector half-space of     */
/* every other generator, one plane at a time (convex polygon clipping of each */
/* face, the cut polygon becomes a new face).                                  */
/* ------------------------------------------------------------------------ */

#define VMAX_FACES 160
#define VMAX_FV 24

typedef struct {
    double n[3];      /* unit outward normal */
    double c;         /* plane n.x = c */
    int64_t nbr;      /* neighbour generator id, or -1-w for box wall w */
    int nv;
    double v[VMAX_FV][3];
} vface;

typedef struct {
    int nf;
    vface f[VMAX_FACES];
    int overflow;
} vpoly;

static void poly_box(vpoly *P, const double *box)
{
    static const int ax[6] = {0, 0, 1, 1, 2, 2};
    P->nf = 6;
    P->overflow = 0;
    double lo[3] = {box[0], box[2], box[4]}, hi[3] = {box[1], box[3], box[5]};
    /* corners indexed by bits (x,y,z) */
    double cc[8][3];
    for (int i = 0; i < 8; ++i) {
        cc[i][0] = (i & 1) ? hi[0] : lo[0];
        cc[i][1] = (i & 2) ? hi[1] : lo[1];
        cc[i][2] = (i & 4) ? hi[2] : lo[2];
    }
    /* faces: -x, +x, -y, +y, -z, +z with CCW loops seen from outside */
    static const int loops[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                    {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    for (int w = 0; w < 6; ++w) {
        vface *F = &P->f[w];
        memset(F->n, 0, sizeof F->n);
        F->n[ax[w]] = (w & 1) ? 1.0 : -1.0;
        F->c = (w & 1) ? hi[ax[w]] : -lo[ax[w]];
        F->nbr = -1 - w;
        F->nv = 4;
        for (int k = 0; k < 4; ++k) memcpy(F->v[k], cc[loops[w][k]], sizeof(double) * 3);
    }
}

/* Clip by n.x <= c (n unit).  eps: distance below which a vertex counts as on the plane. */
static void poly_clip(vpoly *P, const double *n, double c, int64_t nbr, double eps)
{
    double cut[VMAX_FACES * 2][3];
    int ncut = 0;
    int any_out = 0;
    for (int f = 0; f < P->nf && !any_out; ++f)
        for (int k = 0; k < P->f[f].nv; ++k)
            if (dot3(n, P->f[f].v[k]) - c > eps) { any_out = 1; break; }
    if (!any_out) return;
    int nf = 0;
    for (int f = 0; f < P->nf; ++f) {
        vface *F = &P->f[f];
        double out[VMAX_FV][3];
        int no = 0;
        for (int k = 0; k < F->nv; ++k) {
            const double *a = F->v[k], *b = F->v[(k + 1) % F->nv];
            double da = dot3(n, a) - c, db = dot3(n, b) - c;
            int ina = da <= eps;
            if (ina) {
                if (no < VMAX_FV) memcpy(out[no++], a, sizeof(double) * 3); else P->overflow = 1;
                if (fabs(da) <= eps && ncut < VMAX_FACES * 2) memcpy(cut[ncut++], a, sizeof(double) * 3);
            }
            if ((da < -eps && db > eps) || (da > eps && db < -eps)) {
                double t = da / (da - db);
                double x[3] = {a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]), a[2] + t * (b[2] - a[2])};
                if (no < VMAX_FV) memcpy(out[no++], x, sizeof(double) * 3); else P->overflow = 1;
                if (ncut < VMAX_FACES * 2) memcpy(cut[ncut++], x, sizeof(double) * 3);
            }
        }
        if (no >= 3) {
            vface *G = &P->f[nf++];
            if (G != F) *G = *F;
            G->nv = no;
            memcpy(G->v, out, sizeof(double) * 3 * no);
        }
    }
    P->nf = nf;
    /* de-duplicate cut points */
    double uniq[VMAX_FACES * 2][3];
    int nu = 0;
    for (int i = 0; i < ncut; ++i) {
        int dup = 0;
        for (int j = 0; j < nu && !dup; ++j) {
            double d[3] = {cut[i][0] - uniq[j][0], cut[i][1] - uniq[j][1], cut[i][2] - uniq[j][2]};
            if (dot3(d, d) <= 4.0 * eps * eps) dup = 1;
        }
        if (!dup) memcpy(uniq[nu++], cut[i], sizeof(double) * 3);
    }
    if (nu < 3) return;
    if (nu > VMAX_FV || P->nf >= VMAX_FACES) { P->overflow = 1; return; }
    /* order counter-clockwise about n, seen from outside */
    double ctr[3] = {0, 0, 0};
    for (int i = 0; i < nu; ++i) for (int d = 0; d < 3; ++d) ctr[d] += uniq[i][d] / nu;
    double u[3], tmp[3] = {1, 0, 0};
    if (fabs(n[0]) > 0.9) { tmp[0] = 0; tmp[1] = 1; }
    cross3(n, tmp, u);
    double lu = sqrt(dot3(u, u));
    for (int d = 0; d < 3; ++d) u[d] /= lu;
    double v[3];
    cross3(n, u, v);
    double ang[VMAX_FACES * 2];
    for (int i = 0; i < nu; ++i) {
        double r[3] = {uniq[i][0] - ctr[0], uniq[i][1] - ctr[1], uniq[i][2] - ctr[2]};
        ang[i] = atan2(dot3(r, v), dot3(r, u));
    }
    for (int i = 1; i < nu; ++i) {                 /* insertion sort by angle */
        double a = ang[i], x[3];
        memcpy(x, uniq[i], sizeof x);
        int j = i - 1;
        while (j >= 0 && ang[j] > a) { ang[j + 1] = ang[j]; memcpy(uniq[j + 1], uniq[j], sizeof x); --j; }
        ang[j + 1] = a;
        memcpy(uniq[j + 1], x, sizeof x);
    }
    vface *N = &P->f[P->nf++];
    memcpy(N->n, n, sizeof N->n);
    N->c = c;
    N->nbr = nbr;
    N->nv = nu;
    memcpy(N->v, uniq, sizeof(double) * 3 * nu);
}

static double poly_rmax(const vpoly *P, const double *g)
{
    double r2 = 0.0;
    for (int f = 0; f < P->nf; ++f)
        for (int k = 0; k < P->f[f].nv; ++k) {
            double d[3] = {P->f[f].v[k][0] - g[0], P->f[f].v[k][1] - g[1], P->f[f].v[k][2] - g[2]};
            double q = dot3(d, d);
            if (q > r2) r2 = q;
        }
    return sqrt(r2);
}

static double face_area(const vface *F)
{
    double s[3] = {0, 0, 0};
    for (int k = 1; k + 1 < F->nv; ++k) {
        double a[3] = {F->v[k][0] - F->v[0][0], F->v[k][1] - F->v[0][1], F->v[k][2] - F->v[0][2]};
        double b[3] = {F->v[k + 1][0] - F->v[0][0], F->v[k + 1][1] - F->v[0][1], F->v[k + 1][2] - F->v[0][2]};
        double c[3];
        cross3(a, b, c);
        s[0] += c[0]; s[1] += c[1]; s[2] += c[2];
    }
    return 0.5 * dot3(s, F->n);
}

/* Build cells `cells[0..ncells)` of the generator set.  Per cell c, outputs go
 * to slot c: up to max_faces faces and max_fv face vertices.
 * nface_out[c], nfv_out[c]: counts (-1 on overflow); face_nbr, face_normal (3),
 * face_nv, verts (3 per face vertex), volume[c].  Returns the number of cells
 * that overflowed. */
int64_t orc_voronoi_cells(int64_t ngen, const double *gx, const double *gy, const double *gz,
                          const double *box, int64_t ncells, const int64_t *cells, int max_faces,
                          int max_fv, int64_t *nface_out, int64_t *nfv_out, int64_t *face_nbr,
                          double *face_normal, int64_t *face_nv, double *verts, double *volume,
                          int nthreads)
{
    double L = fmax(box[1] - box[0], fmax(box[3] - box[2], box[5] - box[4]));
    double eps = 1e-13 * L;
    int64_t nover = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(+ : nover)
    for (int64_t ci = 0; ci < ncells; ++ci) {
        int64_t j = cells[ci];
        double g[3] = {gx[j], gy[j], gz[j]};
        vpoly *P = (vpoly *)malloc(sizeof(vpoly));
        poly_box(P, box);
        double rmax = poly_rmax(P, g);
        for (int64_t k = 0; k < ngen; ++k) {
            if (k == j) continue;
            double d[3] = {gx[k] - g[0], gy[k] - g[1], gz[k] - g[2]};
            double dd = sqrt(dot3(d, d));
            if (dd == 0.0) continue;                 /* coincident generators: no bisector */
            if (0.5 * dd >= rmax + eps) continue;    /* bisector beyond every vertex */
            double n[3] = {d[0] / dd, d[1] / dd, d[2] / dd};
            double mid[3] = {0.5 * (gx[k] + g[0]), 0.5 * (gy[k] + g[1]), 0.5 * (gz[k] + g[2])};
            int nf0 = P->nf;
            (void)nf0;
            poly_clip(P, n, dot3(n, mid), k, eps);
            rmax = poly_rmax(P, g);
        }
        int64_t fo = ci * (int64_t)max_faces, vo = ci * (int64_t)max_fv;
        int64_t nfv = 0;
        int ok = !P->overflow && P->nf <= max_faces;
        for (int f = 0; ok && f < P->nf; ++f) nfv += P->f[f].nv;
        if (nfv > max_fv) ok = 0;
        if (!ok) {
            nface_out[ci] = -1;
            nfv_out[ci] = -1;
            nover += 1;
            free(P);
            continue;
        }
        double vol = 0.0;
        int64_t vv = 0;
        for (int f = 0; f < P->nf; ++f) {
            const vface *F = &P->f[f];
            face_nbr[fo + f] = F->nbr;
            memcpy(face_normal + 3 * (fo + f), F->n, sizeof(double) * 3);
            face_nv[fo + f] = F->nv;
            for (int k = 0; k < F->nv; ++k, ++vv) memcpy(verts + 3 * (vo + vv), F->v[k], sizeof(double) * 3);
            vol += (F->c - dot3(F->n, g)) * face_area(F) / 3.0;
        }
        nface_out[ci] = P->nf;
        nfv_out[ci] = nfv;
        volume[ci] = vol;
        free(P);
    }
    return nover;
}

/* ------------------------------------------------------------------------ */
/* Particle-cell pairs                                                       */
/* ------------------------------------------------------------------------ */

/* Euclidean distance from p to the convex polygon (nv vertices, unit normal n). */
static double point_polygon_dist(const double *p, int nv, const double *verts, const double *n)
{
    double r0[3] = {p[0] - verts[0], p[1] - verts[1], p[2] - verts[2]};
    double s = dot3(r0, n);
    double P[3] = {p[0] - s * n[0], p[1] - s * n[1], p[2] - s * n[2]};
    int inside = 1;
    double best2 = INFINITY;
    for (int k = 0; k < nv; ++k) {
        const double *a = verts + 3 * k, *b = verts + 3 * ((k + 1) % nv);
        double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double m[3];
        cross3(e, n, m);
        double ra[3] = {a[0] - P[0], a[1] - P[1], a[2] - P[2]};
        if (dot3(ra, m) < 0.0) inside = 0;
        /* distance from p to segment ab */
        double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
        double ee = dot3(e, e);
        double t = ee > 0.0 ? dot3(ap, e) / ee : 0.0;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        double q[3] = {ap[0] - t * e[0], ap[1] - t * e[1], ap[2] - t * e[2]};
        double d2 = dot3(q, q);
        if (d2 < best2) best2 = d2;
    }
    if (inside) return fabs(s);
    return sqrt(best2);
}

/* Distance from p to the closed convex cell (0 if inside). */
double orc_cell_distance(const double *p, int nface, const int64_t *face_vert_off, const double *verts,
                         const double *normals)
{
    int inside = 1;
    for (int f = 0; f < nface && inside; ++f) {
        const double *v0 = verts + 3 * face_vert_off[f];
        double r[3] = {p[0] - v0[0], p[1] - v0[1], p[2] - v0[2]};
        if (dot3(r, normals + 3 * f) > 0.0) inside = 0;
    }
    if (inside) return 0.0;
    double best = INFINITY;
    for (int f = 0; f < nface; ++f) {
        int64_t a = face_vert_off[f], b = face_vert_off[f + 1];
        double d = point_polygon_dist(p, (int)(b - a), verts + 3 * a, normals + 3 * f);
        if (d < best) best = d;
    }
    return best;
}

/* All pairs (i, j) with dist(x_i, V_j) < 2 h_i, for cells given in CSR form
 * (cell_face_off over faces, face_vert_off over face vertices).  Pass 1
 * (pair_i == NULL) fills count[j]; pass 2 writes pairs of cell j at
 * offset[j].. in ascending i, and near[k] = 1 when |dist - 2h| < 1e-9 h.
 * The sphere test |x_i - g_j| > R_j + 2 h_i (R_j: farthest vertex from g_j) only
 * skips pairs that provably do not meet. */
void orc_find_pairs(int64_t np, const double *x, const double *y, const double *z, const double *h,
                    int64_t ncell, const double *gx, const double *gy, const double *gz,
                    const int64_t *cell_face_off, const int64_t *face_vert_off, const double *verts,
                    const double *normals, int64_t *count, const int64_t *offset, int64_t *pair_i,
                    uint8_t *near, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
    for (int64_t j = 0; j < ncell; ++j) {
        int64_t f0 = cell_face_off[j], f1 = cell_face_off[j + 1];
        double g[3] = {gx[j], gy[j], gz[j]};
        double R2 = 0.0;
        for (int64_t v = face_vert_off[f0]; v < face_vert_off[f1]; ++v) {
            double d[3] = {verts[3 * v] - g[0], verts[3 * v + 1] - g[1], verts[3 * v + 2] - g[2]};
            double q = dot3(d, d);
            if (q > R2) R2 = q;
        }
        double R = sqrt(R2);
        int64_t c = 0;
        for (int64_t i = 0; i < np; ++i) {
            double p[3] = {x[i], y[i], z[i]};
            double d[3] = {p[0] - g[0], p[1] - g[1], p[2] - g[2]};
            double rr = R + 2.0 * h[i] * (1.0 + 1e-12);
            if (dot3(d, d) > rr * rr) continue;
            double dist = orc_cell_distance(p, (int)(f1 - f0), face_vert_off + f0, verts, normals + 3 * f0);
            if (dist < 2.0 * h[i]) {
                if (pair_i) {
                    pair_i[offset[j] + c] = i;
                    near[offset[j] + c] = fabs(dist - 2.0 * h[i]) < 1e-9 * h[i];
                }
                ++c;
            }
        }
        if (!pair_i) count[j] = c;
    }
}

/* w for a list of pairs; cells in CSR form.  OpenMP over pairs. */
void orc_map_exact(int64_t npair, const int64_t *pair_i, const int64_t *pair_j, const double *x,
                   const double *y, const double *z, const double *h, const int64_t *cell_face_off,
                   const int64_t *face_vert_off, const double *verts, const double *normals, double *w,
                   int nthreads)
{
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int64_t k = 0; k < npair; ++k) {
        int64_t i = pair_i[k], j = pair_j[k];
        double p[3] = {x[i], y[i], z[i]};
        int64_t f0 = cell_face_off[j], f1 = cell_face_off[j + 1];
        w[k] = orc_cell_weight(p, h[i], (int)(f1 - f0), face_vert_off + f0, verts, normals + 3 * f0);
    }
}

/* rho_j = (sum over the cell's pairs, in the given (ascending i) order, of m_i w_ij) / V_j */
void orc_cell_density(int64_t ncell, const int64_t *cell_pair_off, const int64_t *pair_i, const double *w,
                      const double *m, const double *volume, double *rho)
{
    for (int64_t j = 0; j < ncell; ++j) {
        double s = 0.0;
        for (int64_t k = cell_pair_off[j]; k < cell_pair_off[j + 1]; ++k) s += m[pair_i[k]] * w[k];
        rho[j] = s / volume[j];
    }
}
