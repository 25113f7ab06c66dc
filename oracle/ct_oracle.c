/*
 * ct_oracle.c -- plain FP64 CPU oracle for CT forward projection y = A x and
 * its adjoint backprojection x = A^T y (Sec. 2.3, Eq. 1 and Eq. 2).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark call this code.  It shares nothing with the CUDA
 * library: its own geometry set-up, its own detector mapping, its own weights.
 * It favours plain loops over speed; OpenMP only splits independent outer loops.
 *
 * Conventions (the paper's Sec. 2.2 and Table 1, with the readings it leaves
 * open stated where they are used):
 *   - world origin at the rotation centre; at theta = 0 the y axis is normal
 *     to the detector and the source sits at (x_src, SAD, z_src);
 *   - detector centre at theta = 0: (-u_ofst, SAD - SDD, -v_ofst); detector
 *     axes e_u = (1,0,0), e_v = (0,0,1), normal n = e_u x e_v = (0,-1,0);
 *   - gantry rotation R = Rz(theta) Rx(phi) Ry(psi) ("order y -> x -> z"),
 *     applied to source, detector centre and detector axes;
 *   - voxel centres ((i-(nx-1)/2) dx + x_ofst, ...) ; voxel = centre +- d/2;
 *   - detector cell centres u_a = (a-(nu-1)/2) du, v_b = (b-(nv-1)/2) dv,
 *     measured from the detector centre along e_u, e_v; a curved detector is a
 *     cylinder of radius D = (c-s).n around the axis through the source along
 *     e_v, with u the arc length;
 *   - taps that fall outside the detector are dropped (zero padding);
 *   - a 2D fan-beam geometry is the single-slice case of the 3D one (Sec. 2.2):
 *     nz = nv = 1, unit slice thickness and unit row height, all z offsets 0.
 *
 * Projectors (Sec. 2.3): 0 voxel-driven (point voxel, bilinear detector
 * interpolation), 1 ray-driven (Siddon line lengths), 2 distance-driven
 * (boundary overlaps), 3 separable footprint SF-TR (trapezoid x rectangle),
 * 4 SF-TT (trapezoid x trapezoid, per-cell amplitude; the cited method's
 * variant for large cone angles).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int kind;          /* 0 fan2d, 1 circ3d, 2 noncirc3d */
    int curved;        /* 0 flat, 1 curved */
    int nx, ny, nz;
    double dx, dy, dz;
    int nu, nv;
    double du, dv;
    int nview;
    /* each array holds nview values (the caller repeats scalars) */
    const double *theta, *phi, *psi, *sad, *sdd, *x_src, *z_src;
    const double *x_ofst, *y_ofst, *z_ofst, *u_ofst, *v_ofst;
    const double *poses; /* NULL, or nview x 12: src, det centre, e_u, e_v */
} og_desc;

typedef struct {
    double s[3], c[3], eu[3], ev[3], n[3];
    double D;   /* (c - s).n : source-to-detector-plane distance / radius */
    double u0;  /* (c - s).e_u */
    double h0;  /* (c - s).e_v */
} og_frame;

enum { OG_VOXEL = 0, OG_RAY = 1, OG_DD = 2, OG_SF = 3, OG_SFTT = 4 };
#define OG_FP_CAP 8192

typedef struct {
    int n;
    int a[OG_FP_CAP], b[OG_FP_CAP];
    double w[OG_FP_CAP];
    int overflow;
} og_fp;

static double dot3(const double *p, const double *q) { return p[0]*q[0] + p[1]*q[1] + p[2]*q[2]; }
static double norm3(const double *p) { return sqrt(dot3(p, p)); }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* effective slice thickness / row height: 1 for the 2D fan beam */
static double eff_dz(const og_desc *g) { return g->kind == 0 ? 1.0 : g->dz; }
static double eff_dv(const og_desc *g) { return g->kind == 0 ? 1.0 : g->dv; }

/* R = Rz(th) Rx(ph) Ry(ps): rotate about y first, then x, then z */
static void rotate(double th, double ph, double ps, const double *in, double *out)
{
    double a[3], b[3];
    a[0] =  cos(ps) * in[0] + sin(ps) * in[2];
    a[1] =  in[1];
    a[2] = -sin(ps) * in[0] + cos(ps) * in[2];
    b[0] = a[0];
    b[1] = cos(ph) * a[1] - sin(ph) * a[2];
    b[2] = sin(ph) * a[1] + cos(ph) * a[2];
    out[0] = cos(th) * b[0] - sin(th) * b[1];
    out[1] = sin(th) * b[0] + cos(th) * b[1];
    out[2] = b[2];
}

static void view_frame(const og_desc *g, int v, og_frame *f)
{
    int two_d = (g->kind == 0);
    if (g->poses) {
        const double *p = g->poses + 12 * (size_t)v;
        for (int m = 0; m < 3; ++m) {
            f->s[m] = p[m]; f->c[m] = p[3 + m]; f->eu[m] = p[6 + m]; f->ev[m] = p[9 + m];
        }
        double nu_ = norm3(f->eu), nv_ = norm3(f->ev);
        for (int m = 0; m < 3; ++m) { f->eu[m] /= nu_; f->ev[m] /= nv_; }
    } else {
        double th = g->theta[v];
        double ph = (g->kind == 2) ? g->phi[v] : 0.0;
        double ps = (g->kind == 2) ? g->psi[v] : 0.0;
        double zs = two_d ? 0.0 : g->z_src[v];
        double vo = two_d ? 0.0 : g->v_ofst[v];
        double s0[3] = { g->x_src[v], g->sad[v], zs };
        double c0[3] = { -g->u_ofst[v], g->sad[v] - g->sdd[v], -vo };
        double eu0[3] = { 1.0, 0.0, 0.0 };
        double ev0[3] = { 0.0, 0.0, 1.0 };
        rotate(th, ph, ps, s0, f->s);
        rotate(th, ph, ps, c0, f->c);
        rotate(th, ph, ps, eu0, f->eu);
        rotate(th, ph, ps, ev0, f->ev);
    }
    /* n = e_u x e_v */
    f->n[0] = f->eu[1] * f->ev[2] - f->eu[2] * f->ev[1];
    f->n[1] = f->eu[2] * f->ev[0] - f->eu[0] * f->ev[2];
    f->n[2] = f->eu[0] * f->ev[1] - f->eu[1] * f->ev[0];
    double cs[3] = { f->c[0] - f->s[0], f->c[1] - f->s[1], f->c[2] - f->s[2] };
    f->D = dot3(cs, f->n);
    f->u0 = dot3(cs, f->eu);
    f->h0 = dot3(cs, f->ev);
}

static void voxel_centre(const og_desc *g, int v, int i, int j, int k, double *X)
{
    X[0] = (i - 0.5 * (g->nx - 1)) * g->dx + g->x_ofst[v];
    X[1] = (j - 0.5 * (g->ny - 1)) * g->dy + g->y_ofst[v];
    X[2] = (g->kind == 0) ? 0.0 : (k - 0.5 * (g->nz - 1)) * g->dz + g->z_ofst[v];
}

/* detector coordinates (u, v) in mm of the ray from the source through X */
static void project(const og_frame *f, int curved, const double *X, double *u, double *v)
{
    double w[3] = { X[0] - f->s[0], X[1] - f->s[1], X[2] - f->s[2] };
    double a = dot3(w, f->eu), b = dot3(w, f->ev), c = dot3(w, f->n);
    if (!curved) {
        *u = f->D * a / c - f->u0;
        *v = f->D * b / c - f->h0;
    } else {
        double rho = sqrt(a * a + c * c);
        *u = f->D * atan2(a, c) - f->u0;
        *v = f->D * b / rho - f->h0;
    }
}

static double cell_u(const og_desc *g, int a) { return (a - 0.5 * (g->nu - 1)) * g->du; }
static double cell_v(const og_desc *g, int b) { return (b - 0.5 * (g->nv - 1)) * eff_dv(g); }

/* world position of detector point (u, v) */
static void det_point(const og_frame *f, int curved, double u, double v, double *P)
{
    if (!curved) {
        for (int m = 0; m < 3; ++m) P[m] = f->c[m] + u * f->eu[m] + v * f->ev[m];
    } else {
        double gam = (f->u0 + u) / f->D;
        for (int m = 0; m < 3; ++m)
            P[m] = f->s[m] + f->D * (cos(gam) * f->n[m] + sin(gam) * f->eu[m]) + (f->h0 + v) * f->ev[m];
    }
}

static double overlap(double lo1, double hi1, double lo2, double hi2)
{
    double d = dmin(hi1, hi2) - dmax(lo1, lo2);
    return d > 0.0 ? d : 0.0;
}

/* antiderivative of the unit-height trapezoid with knots t0<=t1<=t2<=t3 */
static double trap_integral(const double *t, double u)
{
    if (u <= t[0]) return 0.0;
    double rise = 0.5 * (t[1] - t[0]);
    if (u <= t[1]) return (u - t[0]) * (u - t[0]) / (2.0 * (t[1] - t[0]));
    if (u <= t[2]) return rise + (u - t[1]);
    double flat = t[2] - t[1];
    double fall = 0.5 * (t[3] - t[2]);
    if (u <= t[3]) return rise + flat + fall - (t[3] - u) * (t[3] - u) / (2.0 * (t[3] - t[2]));
    return rise + flat + fall;
}

static void sort4(double *t)
{
    for (int p = 1; p < 4; ++p) {
        double key = t[p];
        int q = p - 1;
        while (q >= 0 && t[q] > key) { t[q + 1] = t[q]; --q; }
        t[q + 1] = key;
    }
}

static void fp_push(og_fp *fp, int a, int b, double w)
{
    if (fp->n >= OG_FP_CAP) { fp->overflow = 1; return; }
    fp->a[fp->n] = a; fp->b[fp->n] = b; fp->w[fp->n] = w; fp->n++;
}

/* first and last cell index whose interval [x-0.5, x+0.5] (in cells) meets [lo, hi] */
static void cell_range(double lo_mm, double hi_mm, double d, int n, int *first, int *last)
{
    double c = 0.5 * (n - 1);
    int f = (int)floor(lo_mm / d + c + 0.5);
    int l = (int)floor(hi_mm / d + c + 0.5);
    if (f < 0) f = 0;
    if (l > n - 1) l = n - 1;
    *first = f; *last = l;
}

/* ---------- voxel-driven (Peters 1981): point voxel, bilinear on the detector */
static void fp_voxel(const og_desc *g, const og_frame *f, int v, int i, int j, int k, og_fp *fp)
{
    double X[3], u, vv;
    voxel_centre(g, v, i, j, k, X);
    project(f, g->curved, X, &u, &vv);
    double fu = u / g->du + 0.5 * (g->nu - 1);
    double fv = vv / eff_dv(g) + 0.5 * (g->nv - 1);
    double a0 = floor(fu), b0 = floor(fv);
    double ta = fu - a0, tb = fv - b0;
    /* amplitude: the point mass spread over the ray density at its depth */
    double w[3] = { X[0] - f->s[0], X[1] - f->s[1], X[2] - f->s[2] };
    double r = norm3(w);
    double depth;
    if (!g->curved) depth = dot3(w, f->n);
    else { double a = dot3(w, f->eu), c = dot3(w, f->n); depth = sqrt(a * a + c * c); }
    double amp;
    if (g->kind == 0)
        amp = g->dx * g->dy * r * f->D / (depth * depth * g->du);
    else
        amp = g->dx * g->dy * g->dz * r * f->D * f->D / (depth * depth * depth * g->du * g->dv);
    for (int db = 0; db < 2; ++db) {
        int b = (int)b0 + db;
        double hb = db ? tb : 1.0 - tb;
        if (b < 0 || b >= g->nv || hb == 0.0) continue;
        for (int da = 0; da < 2; ++da) {
            int a = (int)a0 + da;
            double ha = da ? ta : 1.0 - ta;
            if (a < 0 || a >= g->nu || ha == 0.0) continue;
            fp_push(fp, a, b, amp * ha * hb);
        }
    }
}

/* ---------- distance-driven (De Man & Basu 2004): boundary overlaps */
static int dd_main_is_y(const og_frame *f)
{
    double d0 = fabs(f->c[0] - f->s[0]), d1 = fabs(f->c[1] - f->s[1]);
    return d1 >= d0;
}

static void fp_dd(const og_desc *g, const og_frame *f, int v, int i, int j, int k, og_fp *fp)
{
    double X[3], P[3], u1, u2, v1, v2, tmp;
    voxel_centre(g, v, i, j, k, X);
    int my = dd_main_is_y(f);
    double dz = eff_dz(g), dv = eff_dv(g);
    /* transaxial boundary points: +-half width along the non-main axis */
    memcpy(P, X, sizeof P);
    if (my) P[0] = X[0] - 0.5 * g->dx; else P[1] = X[1] - 0.5 * g->dy;
    project(f, g->curved, P, &u1, &tmp);
    memcpy(P, X, sizeof P);
    if (my) P[0] = X[0] + 0.5 * g->dx; else P[1] = X[1] + 0.5 * g->dy;
    project(f, g->curved, P, &u2, &tmp);
    /* axial boundary points */
    memcpy(P, X, sizeof P); P[2] = X[2] - 0.5 * dz;
    project(f, g->curved, P, &tmp, &v1);
    memcpy(P, X, sizeof P); P[2] = X[2] + 0.5 * dz;
    project(f, g->curved, P, &tmp, &v2);
    double ulo = dmin(u1, u2), uhi = dmax(u1, u2);
    double vlo = dmin(v1, v2), vhi = dmax(v1, v2);
    int a0, a1, b0, b1;
    cell_range(ulo, uhi, g->du, g->nu, &a0, &a1);
    cell_range(vlo, vhi, dv, g->nv, &b0, &b1);
    double slab = my ? g->dy : g->dx;
    for (int b = b0; b <= b1; ++b) {
        double vc = cell_v(g, b);
        double ov = overlap(vlo, vhi, vc - 0.5 * dv, vc + 0.5 * dv) / dv;
        if (ov == 0.0) continue;
        for (int a = a0; a <= a1; ++a) {
            double uc = cell_u(g, a);
            double ou = overlap(ulo, uhi, uc - 0.5 * g->du, uc + 0.5 * g->du) / g->du;
            if (ou == 0.0) continue;
            double Q[3], d[3];
            det_point(f, g->curved, uc, vc, Q);
            for (int m = 0; m < 3; ++m) d[m] = Q[m] - f->s[m];
            double L = slab * norm3(d) / fabs(my ? d[1] : d[0]);
            fp_push(fp, a, b, ou * ov * L);
        }
    }
}

/* ---------- separable footprint SF-TR (Long, Fessler & Balter 2010) */
static void fp_sf(const og_desc *g, const og_frame *f, int v, int i, int j, int k, og_fp *fp)
{
    double X[3], P[3], tau[4], v1, v2, tmp;
    voxel_centre(g, v, i, j, k, X);
    double dz = eff_dz(g), dv = eff_dv(g);
    /* transaxial footprint: the four column corners at the voxel's z centre */
    int q = 0;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sy = -1; sy <= 1; sy += 2) {
            P[0] = X[0] + 0.5 * sx * g->dx;
            P[1] = X[1] + 0.5 * sy * g->dy;
            P[2] = X[2];
            project(f, g->curved, P, &tau[q++], &tmp);
        }
    sort4(tau);
    /* axial footprint: the column's end points at the voxel's (x, y) centre */
    memcpy(P, X, sizeof P); P[2] = X[2] - 0.5 * dz;
    project(f, g->curved, P, &tmp, &v1);
    memcpy(P, X, sizeof P); P[2] = X[2] + 0.5 * dz;
    project(f, g->curved, P, &tmp, &v2);
    double vlo = dmin(v1, v2), vhi = dmax(v1, v2);
    /* amplitude: voxel width over the larger transaxial direction cosine of
       the 3D unit ray from the source to the voxel centre */
    double w[3] = { X[0] - f->s[0], X[1] - f->s[1], X[2] - f->s[2] };
    double amp = g->dx * norm3(w) / dmax(fabs(w[0]), fabs(w[1]));
    int a0, a1, b0, b1;
    cell_range(tau[0], tau[3], g->du, g->nu, &a0, &a1);
    cell_range(vlo, vhi, dv, g->nv, &b0, &b1);
    for (int b = b0; b <= b1; ++b) {
        double vc = cell_v(g, b);
        double Fv = overlap(vlo, vhi, vc - 0.5 * dv, vc + 0.5 * dv) / dv;
        if (Fv == 0.0) continue;
        for (int a = a0; a <= a1; ++a) {
            double uc = cell_u(g, a);
            double Fu = (trap_integral(tau, uc + 0.5 * g->du) - trap_integral(tau, uc - 0.5 * g->du)) / g->du;
            if (Fu == 0.0) continue;
            fp_push(fp, a, b, amp * Fu * Fv);
        }
    }
}

/* ---------- separable footprint SF-TT (Long, Fessler & Balter 2010):
   the transaxial trapezoid of SF-TR times an axial trapezoid, with the
   amplitude of each detector cell ("A2": the SF-TR amplitude taken along the
   ray to the cell centre instead of the ray to the voxel centre).  The axial
   trapezoid's knots are the projections of the voxel's two z faces (z -+ dz/2)
   at its transaxial corners nearest to and farthest from the source (least
   and greatest depth (P - s).n), sorted.  The nearest corner is the one
   against the detector normal's transaxial components (x offset -sign(n_x) dx/2,
   likewise y); a component below 1e-7 counts as zero and takes the negative
   side for both corners (the two candidates then lie at the same depth). */
static void fp_sftt(const og_desc *g, const og_frame *f, int v, int i, int j, int k, og_fp *fp)
{
    double X[3], P[3], tau[4], tv[4], depth[4], tmp;
    voxel_centre(g, v, i, j, k, X);
    double dz = eff_dz(g), dv = eff_dv(g);
    int q = 0;
    for (int sx = -1; sx <= 1; sx += 2)
        for (int sy = -1; sy <= 1; sy += 2) {
            P[0] = X[0] + 0.5 * sx * g->dx;
            P[1] = X[1] + 0.5 * sy * g->dy;
            P[2] = X[2];
            project(f, g->curved, P, &tau[q++], &tmp);
        }
    sort4(tau);
    const double eps = 1e-7;
    const int nx_sx = f->n[0] < -eps ? 1 : -1, ny_sy = f->n[1] < -eps ? 1 : -1;  /* nearest */
    const int fx_sx = f->n[0] > eps ? 1 : -1, fy_sy = f->n[1] > eps ? 1 : -1;    /* farthest */
    (void)depth;
    q = 0;
    for (int c = 0; c < 2; ++c) {
        int sx = c ? fx_sx : nx_sx, sy = c ? fy_sy : ny_sy;
        for (int sz = -1; sz <= 1; sz += 2) {
            P[0] = X[0] + 0.5 * sx * g->dx;
            P[1] = X[1] + 0.5 * sy * g->dy;
            P[2] = X[2] + 0.5 * sz * dz;
            project(f, g->curved, P, &tmp, &tv[q++]);
        }
    }
    sort4(tv);
    int a0, a1, b0, b1;
    cell_range(tau[0], tau[3], g->du, g->nu, &a0, &a1);
    cell_range(tv[0], tv[3], dv, g->nv, &b0, &b1);
    for (int b = b0; b <= b1; ++b) {
        double vc = cell_v(g, b);
        double Fv = (trap_integral(tv, vc + 0.5 * dv) - trap_integral(tv, vc - 0.5 * dv)) / dv;
        if (Fv == 0.0) continue;
        for (int a = a0; a <= a1; ++a) {
            double uc = cell_u(g, a);
            double Fu = (trap_integral(tau, uc + 0.5 * g->du) - trap_integral(tau, uc - 0.5 * g->du)) / g->du;
            if (Fu == 0.0) continue;
            double C[3];
            det_point(f, g->curved, uc, vc, C);
            double d[3] = { C[0] - f->s[0], C[1] - f->s[1], C[2] - f->s[2] };
            double amp = g->dx * norm3(d) / dmax(fabs(d[0]), fabs(d[1]));
            fp_push(fp, a, b, amp * Fu * Fv);
        }
    }
}

/* ---------- ray-driven (Siddon 1985) */
/* length of the segment s -> P inside the half-open box [lo, hi) */
static double seg_in_box(const double *s, const double *P, const double *lo, const double *hi)
{
    double d[3] = { P[0] - s[0], P[1] - s[1], P[2] - s[2] };
    double t0 = 0.0, t1 = 1.0;
    for (int m = 0; m < 3; ++m) {
        if (d[m] == 0.0) {
            if (s[m] < lo[m] || s[m] >= hi[m]) return 0.0;
        } else {
            double ta = (lo[m] - s[m]) / d[m], tb = (hi[m] - s[m]) / d[m];
            if (ta > tb) { double t = ta; ta = tb; tb = t; }
            t0 = dmax(t0, ta);
            t1 = dmin(t1, tb);
        }
    }
    return t1 > t0 ? (t1 - t0) * norm3(d) : 0.0;
}

static void voxel_box(const og_desc *g, int v, int i, int j, int k, double *lo, double *hi)
{
    double X[3];
    voxel_centre(g, v, i, j, k, X);
    double h[3] = { 0.5 * g->dx, 0.5 * g->dy, 0.5 * eff_dz(g) };
    for (int m = 0; m < 3; ++m) { lo[m] = X[m] - h[m]; hi[m] = X[m] + h[m]; }
}

/* adjoint side of the ray-driven projector: all cells whose central ray meets
   voxel (i,j,k), with the exact intersection length */
static void fp_ray(const og_desc *g, const og_frame *f, int v, int i, int j, int k, og_fp *fp)
{
    double lo[3], hi[3], P[3];
    voxel_box(g, v, i, j, k, lo, hi);
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int cidx = 0; cidx < 8; ++cidx) {
        double uu, vv;
        P[0] = (cidx & 1) ? hi[0] : lo[0];
        P[1] = (cidx & 2) ? hi[1] : lo[1];
        P[2] = (cidx & 4) ? hi[2] : lo[2];
        project(f, g->curved, P, &uu, &vv);
        umin = dmin(umin, uu); umax = dmax(umax, uu);
        vmin = dmin(vmin, vv); vmax = dmax(vmax, vv);
    }
    if (g->curved) {
        /* on a cylinder v is not extreme at the corners: bound it with the
           nearest and farthest horizontal distance of the box from the axis */
        double ex = dmax(dmax(lo[0] - f->s[0], 0.0), f->s[0] - hi[0]);
        double ey = dmax(dmax(lo[1] - f->s[1], 0.0), f->s[1] - hi[1]);
        double rmin = sqrt(ex * ex + ey * ey);
        double fx = dmax(fabs(lo[0] - f->s[0]), fabs(hi[0] - f->s[0]));
        double fy = dmax(fabs(lo[1] - f->s[1]), fabs(hi[1] - f->s[1]));
        double rmax = sqrt(fx * fx + fy * fy);
        double zl = lo[2] - f->s[2], zh = hi[2] - f->s[2];
        vmax = f->D * zh / (zh > 0.0 ? rmin : rmax) - f->h0;
        vmin = f->D * zl / (zl < 0.0 ? rmin : rmax) - f->h0;
    }
    double dv = eff_dv(g);
    int a0 = (int)ceil(umin / g->du + 0.5 * (g->nu - 1)) - 1;
    int a1 = (int)floor(umax / g->du + 0.5 * (g->nu - 1)) + 1;
    int b0 = (int)ceil(vmin / dv + 0.5 * (g->nv - 1)) - 1;
    int b1 = (int)floor(vmax / dv + 0.5 * (g->nv - 1)) + 1;
    if (a0 < 0) a0 = 0;
    if (b0 < 0) b0 = 0;
    if (a1 > g->nu - 1) a1 = g->nu - 1;
    if (b1 > g->nv - 1) b1 = g->nv - 1;
    for (int b = b0; b <= b1; ++b)
        for (int a = a0; a <= a1; ++a) {
            det_point(f, g->curved, cell_u(g, a), cell_v(g, b), P);
            double L = seg_in_box(f->s, P, lo, hi);
            if (L > 0.0) fp_push(fp, a, b, L);
        }
}

static void footprint(const og_desc *g, const og_frame *f, int proj, int v, int i, int j, int k, og_fp *fp)
{
    fp->n = 0;
    switch (proj) {
    case OG_VOXEL: fp_voxel(g, f, v, i, j, k, fp); break;
    case OG_RAY:   fp_ray(g, f, v, i, j, k, fp); break;
    case OG_DD:    fp_dd(g, f, v, i, j, k, fp); break;
    case OG_SFTT:  fp_sftt(g, f, v, i, j, k, fp); break;
    default:       fp_sf(g, f, v, i, j, k, fp); break;
    }
}

static int cmp_double(const void *p, const void *q)
{
    double a = *(const double *)p, b = *(const double *)q;
    return (a > b) - (a < b);
}

/* Siddon's method: line integral of vol along the segment s -> P.  The plane
   crossings of the three axes are merged in order of the ray parameter; each
   interval between consecutive crossings lies in one voxel, found from its
   midpoint, and contributes (interval length) x (voxel value). */
static void siddon(const og_desc *g, int v, const double *vol, int batch, size_t vstride,
                   const double *s, const double *P, double *alist, double *out)
{
    int n[3] = { g->nx, g->ny, g->kind == 0 ? 1 : g->nz };
    double h[3] = { g->dx, g->dy, eff_dz(g) };
    double off[3] = { g->x_ofst[v], g->y_ofst[v], g->kind == 0 ? 0.0 : g->z_ofst[v] };
    double lo[3], d[3];
    for (int m = 0; m < 3; ++m) {
        lo[m] = off[m] - 0.5 * n[m] * h[m];
        d[m] = P[m] - s[m];
    }
    double amin = 0.0, amax = 1.0;
    for (int m = 0; m < 3; ++m) {
        if (d[m] == 0.0) {
            if (s[m] < lo[m] || s[m] >= lo[m] + n[m] * h[m]) return;
            continue;
        }
        double a0 = (lo[m] - s[m]) / d[m];
        double a1 = (lo[m] + n[m] * h[m] - s[m]) / d[m];
        amin = dmax(amin, dmin(a0, a1));
        amax = dmin(amax, dmax(a0, a1));
    }
    if (amax <= amin) return;
    int cnt = 0;
    alist[cnt++] = amin;
    for (int m = 0; m < 3; ++m) {
        if (d[m] == 0.0) continue;
        for (int p = 0; p <= n[m]; ++p) {
            double a = (lo[m] + p * h[m] - s[m]) / d[m];
            if (a > amin && a < amax) alist[cnt++] = a;
        }
    }
    alist[cnt++] = amax;
    qsort(alist, (size_t)cnt, sizeof(double), cmp_double);
    double len = norm3(d);
    for (int q = 0; q + 1 < cnt; ++q) {
        double da = alist[q + 1] - alist[q];
        if (da <= 0.0) continue;
        double am = 0.5 * (alist[q + 1] + alist[q]);
        int idx[3];
        int ok = 1;
        for (int m = 0; m < 3; ++m) {
            idx[m] = (int)floor((s[m] + am * d[m] - lo[m]) / h[m]);
            if (idx[m] < 0 || idx[m] >= n[m]) ok = 0;
        }
        if (!ok) continue;
        size_t vi = ((size_t)idx[2] * g->ny + idx[1]) * g->nx + idx[0];
        for (int bt = 0; bt < batch; ++bt) out[bt] += da * len * vol[bt * vstride + vi];
    }
}

/* ------------------------------------------------------------------ API */

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int nz_eff(const og_desc *g) { return g->kind == 0 ? 1 : g->nz; }
static int nv_eff(const og_desc *g) { return g->kind == 0 ? 1 : g->nv; }

/* y = A x.  vol: batch x nz x ny x nx, sino: batch x nview x nv x nu (overwritten).
   Returns 0, or 1 when a footprint exceeded the fixed capacity. */
int oracle_forward(const og_desc *g, int proj, const double *vol, double *sino, int batch)
{
    int nz = nz_eff(g), nv = nv_eff(g);
    size_t vstride = (size_t)g->nx * g->ny * nz;
    size_t view_sz = (size_t)nv * g->nu;
    size_t sstride = view_sz * g->nview;
    int err = 0;
    memset(sino, 0, sizeof(double) * sstride * batch);
    if (proj == OG_RAY) {
#pragma omp parallel
        {
            double *alist = (double *)malloc(sizeof(double) * (size_t)(g->nx + g->ny + nz + 8));
            double *acc = (double *)malloc(sizeof(double) * (size_t)batch);
#pragma omp for schedule(dynamic) collapse(2)
            for (int v = 0; v < g->nview; ++v)
                for (int b = 0; b < nv; ++b) {
                    og_frame f;
                    view_frame(g, v, &f);
                    for (int a = 0; a < g->nu; ++a) {
                        double P[3];
                        det_point(&f, g->curved, cell_u(g, a), cell_v(g, b), P);
                        for (int bt = 0; bt < batch; ++bt) acc[bt] = 0.0;
                        siddon(g, v, vol, batch, vstride, f.s, P, alist, acc);
                        for (int bt = 0; bt < batch; ++bt)
                            sino[bt * sstride + (size_t)v * view_sz + (size_t)b * g->nu + a] = acc[bt];
                    }
                }
            free(alist);
            free(acc);
        }
        return 0;
    }
#pragma omp parallel
    {
        og_fp *fp = (og_fp *)malloc(sizeof(og_fp));
        fp->overflow = 0;
#pragma omp for schedule(dynamic)
        for (int v = 0; v < g->nview; ++v) {
            og_frame f;
            view_frame(g, v, &f);
            double *yv = sino + (size_t)v * view_sz;
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < g->ny; ++j)
                    for (int i = 0; i < g->nx; ++i) {
                        size_t vi = ((size_t)k * g->ny + j) * g->nx + i;
                        footprint(g, &f, proj, v, i, j, k, fp);
                        for (int t = 0; t < fp->n; ++t)
                            for (int bt = 0; bt < batch; ++bt)
                                yv[bt * sstride + (size_t)fp->b[t] * g->nu + fp->a[t]] +=
                                    fp->w[t] * vol[bt * vstride + vi];
                    }
        }
        if (fp->overflow) {
#pragma omp atomic write
            err = 1;
        }
        free(fp);
    }
    return err;
}

/* x[sel] = (A^T y)[sel] for the listed flat voxel indices (k*ny + j)*nx + i;
   out: batch x nsel.  nsel < 0 means every voxel (out: batch x volume). */
int oracle_back_voxels(const og_desc *g, int proj, const double *sino, int batch,
                       long long nsel, const long long *sel, double *out)
{
    int nz = nz_eff(g), nv = nv_eff(g);
    size_t view_sz = (size_t)nv * g->nu;
    size_t sstride = view_sz * g->nview;
    long long total = nsel < 0 ? (long long)g->nx * g->ny * nz : nsel;
    og_frame *frames = (og_frame *)malloc(sizeof(og_frame) * (size_t)g->nview);
    int err = 0;
    for (int v = 0; v < g->nview; ++v) view_frame(g, v, &frames[v]);
#pragma omp parallel
    {
        og_fp *fp = (og_fp *)malloc(sizeof(og_fp));
        double *acc = (double *)malloc(sizeof(double) * (size_t)batch);
        fp->overflow = 0;
#pragma omp for schedule(dynamic, 64)
        for (long long q = 0; q < total; ++q) {
            long long vi = nsel < 0 ? q : sel[q];
            int i = (int)(vi % g->nx);
            int j = (int)((vi / g->nx) % g->ny);
            int k = (int)(vi / ((long long)g->nx * g->ny));
            for (int bt = 0; bt < batch; ++bt) acc[bt] = 0.0;
            for (int v = 0; v < g->nview; ++v) {
                footprint(g, &frames[v], proj, v, i, j, k, fp);
                const double *yv = sino + (size_t)v * view_sz;
                for (int t = 0; t < fp->n; ++t)
                    for (int bt = 0; bt < batch; ++bt)
                        acc[bt] += fp->w[t] * yv[bt * sstride + (size_t)fp->b[t] * g->nu + fp->a[t]];
            }
            for (int bt = 0; bt < batch; ++bt) out[(size_t)bt * total + q] = acc[bt];
        }
        if (fp->overflow) {
#pragma omp atomic write
            err = 1;
        }
        free(fp);
        free(acc);
    }
    free(frames);
    return err;
}

/* x = A^T y over the whole volume (overwritten): batch x nz x ny x nx */
int oracle_back(const og_desc *g, int proj, const double *sino, double *vol, int batch)
{
    return oracle_back_voxels(g, proj, sino, batch, -1, NULL, vol);
}

/* footprint of one voxel in one view: cells (a, b) with weights; returns the
   count (or -1 when it exceeds cap) */
int oracle_footprint(const og_desc *g, int proj, int v, int i, int j, int k,
                     int cap, int *a, int *b, double *w)
{
    og_frame f;
    og_fp *fp = (og_fp *)malloc(sizeof(og_fp));
    fp->overflow = 0;
    view_frame(g, v, &f);
    footprint(g, &f, proj, v, i, j, k, fp);
    int n = fp->n;
    if (fp->overflow || n > cap) n = -1;
    else
        for (int t = 0; t < n; ++t) { a[t] = fp->a[t]; b[t] = fp->b[t]; w[t] = fp->w[t]; }
    free(fp);
    return n;
}

/* the view's frame: s, c, e_u, e_v, n (3 each), D, u0, h0 */
void oracle_frame(const og_desc *g, int v, double *out18)
{
    og_frame f;
    view_frame(g, v, &f);
    memcpy(out18, f.s, 3 * sizeof(double));
    memcpy(out18 + 3, f.c, 3 * sizeof(double));
    memcpy(out18 + 6, f.eu, 3 * sizeof(double));
    memcpy(out18 + 9, f.ev, 3 * sizeof(double));
    memcpy(out18 + 12, f.n, 3 * sizeof(double));
    out18[15] = f.D; out18[16] = f.u0; out18[17] = f.h0;
}

/* detector (u, v) in mm of world point X in view v */
void oracle_project(const og_desc *g, int v, const double *X, double *uv)
{
    og_frame f;
    view_frame(g, v, &f);
    project(&f, g->curved, X, &uv[0], &uv[1]);
}

/* world position of the centre of cell (a, b) in view v */
void oracle_cell_point(const og_desc *g, int v, int a, int b, double *P)
{
    og_frame f;
    view_frame(g, v, &f);
    det_point(&f, g->curved, cell_u(g, a), cell_v(g, b), P);
}

/* ------------------------------------------------------------------ "recon" mode
 * Filtered backprojection (Sec. 2.3: the "recon" mode backprojection carries
 * a depth-dependent weighting, after Kak & Slaney 2001), written in the
 * detector's own coordinates.  Per view: D = source-detector distance (flat)
 * or detector radius (curved); (u_p, v_p) = detector coordinates measured
 * from the principal point (the foot of the source's perpendicular), i.e.
 * u + u0, v + h0; R = (O - s).n, the source's distance to the rotation centre
 * O = 0 along the principal ray; dbeta = the view's share of the gantry angle.
 *   flat:   p_w = p D / sqrt(D^2 + u_p^2 + v_p^2)
 *           q(u_m) = du sum_n p_w(u_n) h(u_m - u_n),
 *           h(0) = 1/(8 du^2), h(k du) = -1/(2 pi^2 k^2 du^2) for odd k, 0 for even k
 *           f(X) = sum_views dbeta R D / ((X - s).n)^2 q(u(X), v(X))
 *   curved: p_w = p R cos(gamma_p) D / sqrt(D^2 + v_p^2), gamma_p = u_p / D
 *           q(u_m) = dg sum_n p_w(u_n) h_c(u_m - u_n), dg = du / D,
 *           h_c(0) = 1/(8 dg^2), h_c(k dg) = -1/(2 pi^2 sin^2(k dg)) for odd k
 *           f(X) = sum_views dbeta / rho^2 q(u(X), v(X)), rho^2 = ((X-s).e_u)^2 + ((X-s).n)^2
 * with bilinear interpolation of q at the projection of the voxel centre
 * (taps off the detector dropped).  h is half the band-limited ramp of
 * Kak & Slaney (the backprojection runs over the full 2 pi).
 */
static const double OG_PI = 3.14159265358979323846;

/* the view's share of the gantry angle: half the angular gap to the
   neighbouring views on the circle (2 pi / nview when there are no angles) */
static double recon_dbeta(const og_desc *g, int v)
{
    if (g->poses || g->nview == 1) return 2.0 * OG_PI / g->nview;
    double th = fmod(g->theta[v], 2.0 * OG_PI);
    if (th < 0) th += 2.0 * OG_PI;
    double prev = 2.0 * OG_PI, next = 2.0 * OG_PI;
    for (int w = 0; w < g->nview; ++w) {
        if (w == v) continue;
        double t = fmod(g->theta[w], 2.0 * OG_PI);
        if (t < 0) t += 2.0 * OG_PI;
        double fwd = fmod(t - th + 4.0 * OG_PI, 2.0 * OG_PI);  /* gap going forward */
        double bwd = fmod(th - t + 4.0 * OG_PI, 2.0 * OG_PI);
        if (fwd > 0 && fwd < next) next = fwd;
        if (bwd > 0 && bwd < prev) prev = bwd;
    }
    return 0.5 * (prev + next);
}

static double recon_kernel(const og_desc *g, const og_frame *f, int k)
{
    if (k == 0) {
        double st = g->curved ? g->du / f->D : g->du;
        return 1.0 / (8.0 * st * st);
    }
    if (k % 2 == 0) return 0.0;
    if (g->curved) {
        double s = sin(k * g->du / f->D);
        return -1.0 / (2.0 * OG_PI * OG_PI * s * s);
    }
    return -1.0 / (2.0 * OG_PI * OG_PI * (double)k * k * g->du * g->du);
}

/* q = ramp-filtered, pre-weighted projections: in, out batch x nview x nv x nu */
int oracle_ramp_filter(const og_desc *g, const double *in, double *out, int batch)
{
    int nv = nv_eff(g);
    size_t view_sz = (size_t)nv * g->nu, sstride = view_sz * g->nview;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int v = 0; v < g->nview; ++v)
        for (int b = 0; b < nv; ++b) {
            og_frame f;
            view_frame(g, v, &f);
            double R = -dot3(f.s, f.n);
            double vp = (g->kind == 0) ? 0.0 : cell_v(g, b) + f.h0;
            double *pw = (double *)malloc(sizeof(double) * (size_t)g->nu);
            double *kern = (double *)malloc(sizeof(double) * (size_t)g->nu);
            for (int k = 0; k < g->nu; ++k) kern[k] = recon_kernel(g, &f, k);
            double step = g->curved ? g->du / f.D : g->du;
            for (int bt = 0; bt < batch; ++bt) {
                const double *row = in + bt * sstride + (size_t)v * view_sz + (size_t)b * g->nu;
                double *orow = out + bt * sstride + (size_t)v * view_sz + (size_t)b * g->nu;
                for (int n = 0; n < g->nu; ++n) {
                    double up = cell_u(g, n) + f.u0;
                    double w;
                    if (g->curved)
                        w = R * cos(up / f.D) * f.D / sqrt(f.D * f.D + vp * vp);
                    else
                        w = f.D / sqrt(f.D * f.D + up * up + vp * vp);
                    pw[n] = row[n] * w;
                }
                for (int m = 0; m < g->nu; ++m) {
                    double s = 0.0;
                    for (int n = 0; n < g->nu; ++n) s += pw[n] * kern[m > n ? m - n : n - m];
                    orow[m] = step * s;
                }
            }
            free(pw);
            free(kern);
        }
    return 0;
}

/* Recon-mode interpolation weights of the footprint projectors: the
   projector's transaxial and axial footprints, each normalised to a unit
   total (so they act as an interpolation kernel, like the bilinear hat):
     DD: (overlap with [u-, u+]) / (u+ - u-) x (overlap with [v-, v+]) / (v+ - v-)
     SF: (integral of the trapezoid over the cell) / (its area) x the same axial factor
   with the boundary points / corners of fp_dd / fp_sf. */
static void recon_fp(const og_desc *g, const og_frame *f, int proj, int v, int i, int j, int k, og_fp *fp)
{
    double X[3], P[3], tau[4], v1, v2, tmp;
    fp->n = 0;
    voxel_centre(g, v, i, j, k, X);
    double dz = eff_dz(g), dv = eff_dv(g);
    if (proj == OG_DD) {
        int my = dd_main_is_y(f);
        memcpy(P, X, sizeof P);
        if (my) P[0] = X[0] - 0.5 * g->dx; else P[1] = X[1] - 0.5 * g->dy;
        project(f, g->curved, P, &tau[0], &tmp);
        memcpy(P, X, sizeof P);
        if (my) P[0] = X[0] + 0.5 * g->dx; else P[1] = X[1] + 0.5 * g->dy;
        project(f, g->curved, P, &tau[3], &tmp);
        if (tau[0] > tau[3]) { tmp = tau[0]; tau[0] = tau[3]; tau[3] = tmp; }
        tau[1] = tau[0];
        tau[2] = tau[3];
    } else {
        int q = 0;
        for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) {
                P[0] = X[0] + 0.5 * sx * g->dx;
                P[1] = X[1] + 0.5 * sy * g->dy;
                P[2] = X[2];
                project(f, g->curved, P, &tau[q++], &tmp);
            }
        sort4(tau);
    }
    memcpy(P, X, sizeof P); P[2] = X[2] - 0.5 * dz;
    project(f, g->curved, P, &tmp, &v1);
    memcpy(P, X, sizeof P); P[2] = X[2] + 0.5 * dz;
    project(f, g->curved, P, &tmp, &v2);
    double vlo = dmin(v1, v2), vhi = dmax(v1, v2);
    double area = 0.5 * (tau[3] + tau[2] - tau[1] - tau[0]), height = vhi - vlo;
    int a0, a1, b0, b1;
    cell_range(tau[0], tau[3], g->du, g->nu, &a0, &a1);
    cell_range(vlo, vhi, dv, g->nv, &b0, &b1);
    for (int b = b0; b <= b1; ++b) {
        double vc = cell_v(g, b);
        double Fv = overlap(vlo, vhi, vc - 0.5 * dv, vc + 0.5 * dv) / height;
        if (Fv == 0.0) continue;
        for (int a = a0; a <= a1; ++a) {
            double uc = cell_u(g, a);
            double Fu = (trap_integral(tau, uc + 0.5 * g->du) - trap_integral(tau, uc - 0.5 * g->du)) / area;
            if (Fu == 0.0) continue;
            fp_push(fp, a, b, Fu * Fv);
        }
    }
}

/* x = recon-mode backprojection of filtered projections q (Sec. 2.3):
   vol batch x nz x ny x nx.  proj: OG_VOXEL (bilinear interpolation) or
   OG_DD / OG_SF (their normalised footprints, recon_fp). */
int oracle_back_recon_proj(const og_desc *g, int proj, const double *q, double *vol, int batch);

int oracle_back_recon(const og_desc *g, const double *q, double *vol, int batch)
{
    return oracle_back_recon_proj(g, OG_VOXEL, q, vol, batch);
}

int oracle_back_recon_proj(const og_desc *g, int proj, const double *q, double *vol, int batch)
{
    int nz = nz_eff(g), nv = nv_eff(g);
    size_t view_sz = (size_t)nv * g->nu, sstride = view_sz * g->nview;
    size_t vstride = (size_t)g->nx * g->ny * nz;
    og_frame *frames = (og_frame *)malloc(sizeof(og_frame) * (size_t)g->nview);
    double *dbeta = (double *)malloc(sizeof(double) * (size_t)g->nview);
    for (int v = 0; v < g->nview; ++v) {
        view_frame(g, v, &frames[v]);
        dbeta[v] = recon_dbeta(g, v);
    }
    long long total = (long long)vstride;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long vi = 0; vi < total; ++vi) {
        int i = (int)(vi % g->nx), j = (int)((vi / g->nx) % g->ny), k = (int)(vi / ((long long)g->nx * g->ny));
        for (int bt = 0; bt < batch; ++bt) vol[bt * vstride + vi] = 0.0;
        for (int v = 0; v < g->nview; ++v) {
            const og_frame *f = &frames[v];
            double X[3], u, vv;
            voxel_centre(g, v, i, j, k, X);
            project(f, g->curved, X, &u, &vv);
            double w[3] = { X[0] - f->s[0], X[1] - f->s[1], X[2] - f->s[2] };
            double a = dot3(w, f->eu), c = dot3(w, f->n);
            double W = g->curved ? dbeta[v] / (a * a + c * c) : dbeta[v] * (-dot3(f->s, f->n)) * f->D / (c * c);
            if (proj != OG_VOXEL) {
                og_fp *fp = (og_fp *)malloc(sizeof(og_fp));
                fp->overflow = 0;
                recon_fp(g, f, proj, v, i, j, k, fp);
                for (int t = 0; t < fp->n; ++t)
                    for (int bt = 0; bt < batch; ++bt)
                        vol[bt * vstride + vi] += W * fp->w[t] *
                            q[bt * sstride + (size_t)v * view_sz + (size_t)fp->b[t] * g->nu + fp->a[t]];
                free(fp);
                continue;
            }
            double fa = u / g->du + 0.5 * (g->nu - 1);
            double fb = (g->kind == 0) ? 0.0 : vv / g->dv + 0.5 * (nv - 1);
            int a0 = (int)floor(fa), b0 = (int)floor(fb);
            double ta = fa - a0, tb = fb - b0;
            for (int db = 0; db < 2; ++db) {
                int b = b0 + db;
                double hb = db ? tb : 1.0 - tb;
                if (b < 0 || b >= nv || hb == 0.0) continue;
                for (int da = 0; da < 2; ++da) {
                    int aa = a0 + da;
                    double ha = da ? ta : 1.0 - ta;
                    if (aa < 0 || aa >= g->nu || ha == 0.0) continue;
                    for (int bt = 0; bt < batch; ++bt)
                        vol[bt * vstride + vi] += W * ha * hb * q[bt * sstride + (size_t)v * view_sz + (size_t)b * g->nu + aa];
                }
            }
        }
    }
    free(frames);
    free(dbeta);
    return 0;
}

/* the view's share of the gantry angle, as used by the recon mode */
double oracle_recon_dbeta(const og_desc *g, int v) { return recon_dbeta(g, v); }
