// ct_capi.cpp -- the C ABI of libctproj: geometry set-up in FP64 (Sec. 2.2,
// Table 1), argument validation, and dispatch of the projector kernels
// (Sec. 2.3).  No call here synchronises the device; only geometry creation
// and destruction allocate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ctproj.h"
#include "ct_geometry.h"
#include "ct_launch.h"
#include "ct_types.h"

using ctp::CtGrid;
using ctp::CtView;


namespace {

thread_local std::string g_err;

ct_status fail(ct_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

struct Vec3 {
    double x, y, z;
};
Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
Vec3 operator*(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
Vec3 cross(Vec3 a, Vec3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double norm(Vec3 a) { return std::sqrt(dot(a, a)); }

struct Mat3 {
    double m[3][3];
    Vec3 operator*(Vec3 v) const {
        return {m[0][0] * v.x + m[0][1] * v.y + m[0][2] * v.z, m[1][0] * v.x + m[1][1] * v.y + m[1][2] * v.z,
                m[2][0] * v.x + m[2][1] * v.y + m[2][2] * v.z};
    }
    Mat3 operator*(const Mat3 &o) const {
        Mat3 r{};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) r.m[i][j] += m[i][k] * o.m[k][j];
        return r;
    }
};
Mat3 rot_z(double t) { return {{{std::cos(t), -std::sin(t), 0}, {std::sin(t), std::cos(t), 0}, {0, 0, 1}}}; }
Mat3 rot_x(double t) { return {{{1, 0, 0}, {0, std::cos(t), -std::sin(t)}, {0, std::sin(t), std::cos(t)}}}; }
Mat3 rot_y(double t) { return {{{std::cos(t), 0, std::sin(t)}, {0, 1, 0}, {-std::sin(t), 0, std::cos(t)}}}; }

// a per-view parameter: NULL -> 0, length 1 -> shared, length nview -> per view
struct Param {
    const double *p;
    int n;
    const char *name;
    double at(int v) const { return p == nullptr ? 0.0 : (n == 1 ? p[0] : p[v]); }
};

bool param_ok(const Param &q, int nview, std::string &why) {
    if (q.p == nullptr) return true;
    if (q.n == 1 || q.n == nview) return true;
    why = std::string(q.name) + ": length " + std::to_string(q.n) + " is neither 1 nor nview=" +
          std::to_string(nview);
    return false;
}

// Source, detector centre and detector axes of view v (Sec. 2.2, Table 1).
void view_pose(const ct_geometry_desc *d, int v, const Param P[], Vec3 &s, Vec3 &c, Vec3 &eu, Vec3 &ev) {
    const bool two_d = d->kind == CT_FAN2D;
    if (d->poses) {
        const double *p = d->poses + 12 * (size_t)v;
        s = {p[0], p[1], p[2]};
        c = {p[3], p[4], p[5]};
        eu = {p[6], p[7], p[8]};
        ev = {p[9], p[10], p[11]};
        eu = (1.0 / norm(eu)) * eu;
        ev = (1.0 / norm(ev)) * ev;
        return;
    }
    // P: theta phi psi sad sdd x_src z_src x_ofst y_ofst z_ofst u_ofst v_ofst
    const double th = P[0].at(v);
    const double ph = d->kind == CT_NONCIRC3D ? P[1].at(v) : 0.0;
    const double ps = d->kind == CT_NONCIRC3D ? P[2].at(v) : 0.0;
    const double sad = P[3].at(v), sdd = P[4].at(v);
    const Mat3 R = rot_z(th) * rot_x(ph) * rot_y(ps);  // rotation order y -> x -> z
    const Vec3 s0{P[5].at(v), sad, two_d ? 0.0 : P[6].at(v)};
    const Vec3 c0{-P[10].at(v), sad - sdd, two_d ? 0.0 : -P[11].at(v)};
    s = R * s0;
    c = R * c0;
    eu = R * Vec3{1, 0, 0};
    ev = R * Vec3{0, 0, 1};
}

// Recon mode (FBP): each view's share of the gantry angle, half the angular
// gaps to the nearest distinct view angles on either side (2 pi / nview for
// an equally spaced full scan; 2 pi / nview for pose-given geometries).
std::vector<double> recon_dbetas(const ct_geometry_desc *d, const Param P[]) {
    const double two_pi = 2.0 * M_PI;
    std::vector<double> out(d->nview, two_pi / d->nview);
    if (d->poses || d->nview == 1) return out;
    std::vector<double> th(d->nview);
    for (int v = 0; v < d->nview; ++v) {
        double t = std::fmod(P[0].at(v), two_pi);
        th[v] = t < 0 ? t + two_pi : t;
    }
    std::vector<double> u(th);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    const size_t m = u.size();
    for (int v = 0; v < d->nview; ++v) {
        const size_t i = std::lower_bound(u.begin(), u.end(), th[v]) - u.begin();
        const double next = m == 1 ? two_pi : (i + 1 < m ? u[i + 1] - u[i] : u[0] + two_pi - u[i]);
        const double prev = m == 1 ? two_pi : (i > 0 ? u[i] - u[i - 1] : u[i] + two_pi - u[m - 1]);
        out[v] = 0.5 * (prev + next);
    }
    return out;
}

}  // namespace

void ctp::set_last_error(const std::string &msg) { g_err = msg; }

namespace ctp {
// Host-side check that p is device (or managed) memory: a host or unknown
// pointer is rejected with CT_ERR_INVALID_ARG before any kernel is launched.
ct_status check_device_ptr(const void *p, const char *what) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CT_ERR_INVALID_ARG, std::string(what) + ": not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(CT_ERR_INVALID_ARG, std::string(what) + ": not device memory");
    return CT_OK;
}
}  // namespace ctp

extern "C" {

const char *ct_last_error(void) { return g_err.c_str(); }

const char *ct_version(void) { return "ctproj 0.1 (sm_103a)"; }

ct_status ct_geometry_create(const ct_geometry_desc *d, ct_geometry **out) {
    if (!d || !out) return fail(CT_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (d->kind < CT_FAN2D || d->kind > CT_NONCIRC3D) return fail(CT_ERR_INVALID_ARG, "unknown geometry kind");
    if (d->det != CT_DET_FLAT && d->det != CT_DET_CURVED) return fail(CT_ERR_INVALID_ARG, "unknown detector kind");
    if (d->det == CT_DET_CURVED && d->kind == CT_NONCIRC3D)
        return fail(CT_ERR_UNSUPPORTED, "curved detectors exist for fan-beam and circular geometries only");
    const bool two_d = d->kind == CT_FAN2D;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nu < 1 || d->nv < 1 || d->nview < 1)
        return fail(CT_ERR_INVALID_ARG, "sizes must be >= 1");
    if (two_d && (d->nz != 1 || d->nv != 1)) return fail(CT_ERR_INVALID_ARG, "fan-beam geometry needs nz = nv = 1");
    if (!(d->dx > 0 && d->dy > 0 && d->du > 0) || (!two_d && !(d->dz > 0 && d->dv > 0)))
        return fail(CT_ERR_INVALID_ARG, "voxel and cell sizes must be > 0");
    if (d->nx > 65536 || d->ny > 65536 || d->nz > 65536 || d->nu > 65536 || d->nv > 65536 ||
        d->nview > (1 << 24))
        return fail(CT_ERR_INVALID_ARG, "size out of range");
    if (d->poses && d->kind != CT_NONCIRC3D) return fail(CT_ERR_INVALID_ARG, "poses need a non-circular geometry");
    const Param P[12] = {{d->theta, d->n_theta, "theta"},    {d->phi, d->n_phi, "phi"},
                         {d->psi, d->n_psi, "psi"},          {d->sad, d->n_sad, "sad"},
                         {d->sdd, d->n_sdd, "sdd"},          {d->x_src, d->n_x_src, "x_src"},
                         {d->z_src, d->n_z_src, "z_src"},    {d->x_ofst, d->n_x_ofst, "x_ofst"},
                         {d->y_ofst, d->n_y_ofst, "y_ofst"}, {d->z_ofst, d->n_z_ofst, "z_ofst"},
                         {d->u_ofst, d->n_u_ofst, "u_ofst"}, {d->v_ofst, d->n_v_ofst, "v_ofst"}};
    std::string why;
    for (const Param &q : P)
        if (!param_ok(q, d->nview, why)) return fail(CT_ERR_INVALID_ARG, why);
    if (!d->poses && (!d->sad || !d->sdd)) return fail(CT_ERR_INVALID_ARG, "sad and sdd are required");
    for (const Param &q : P)
        if (q.p)
            for (int v = 0; v < (q.n == 1 ? 1 : d->nview); ++v)
                if (!std::isfinite(q.p[v])) return fail(CT_ERR_INVALID_ARG, std::string(q.name) + " is not finite");

    ct_geometry *g = new (std::nothrow) ct_geometry();
    if (!g) return fail(CT_ERR_OOM, "host allocation failed");
    g->kind = d->kind;
    g->det = d->det;
    g->nx = d->nx; g->ny = d->ny; g->nz = d->nz;
    g->nu = d->nu; g->nv = d->nv; g->nview = d->nview;
    g->dx = d->dx; g->dy = d->dy;
    g->dz = two_d ? 1.0 : d->dz;   // 2D: unit slice thickness and row height
    g->du = d->du;
    g->dv = two_d ? 1.0 : d->dv;
    const bool curved = d->det == CT_DET_CURVED;
    g->host_views.resize(d->nview);
    const std::vector<double> dbeta = recon_dbetas(d, P);

    for (int v = 0; v < d->nview; ++v) {
        Vec3 s, c, eu, ev;
        view_pose(d, v, P, s, c, eu, ev);
        if (d->poses && std::fabs(dot(eu, ev)) > 1e-6) {
            delete g;
            return fail(CT_ERR_INVALID_ARG, "pose " + std::to_string(v) + ": e_u and e_v are not orthogonal");
        }
        const Vec3 n = cross(eu, ev);
        const Vec3 cs = c - s;
        const double D = dot(cs, n), u0 = dot(cs, eu), h0 = dot(cs, ev);
        if (!(D > 0)) {
            delete g;
            return fail(CT_ERR_INVALID_ARG, "view " + std::to_string(v) + ": detector is not in front of the source");
        }
        const Vec3 X0{-(g->nx - 1) * 0.5 * g->dx + P[7].at(v), -(g->ny - 1) * 0.5 * g->dy + P[8].at(v),
                      two_d ? 0.0 : -(g->nz - 1) * 0.5 * g->dz + P[9].at(v)};
        const Vec3 o = X0 - s;
        CtView &V = g->host_views[v];
        std::memset(&V, 0, sizeof V);
        const double h[3] = {g->dx, g->dy, g->dz};
        const Vec3 axes[3] = {eu, ev, n};
        float *rows[3] = {V.au, V.av, V.an};
        for (int r = 0; r < 3; ++r) {
            rows[r][0] = (float)(h[0] * axes[r].x);
            rows[r][1] = (float)(h[1] * axes[r].y);
            rows[r][2] = (float)(h[2] * axes[r].z);
            rows[r][3] = (float)dot(o, axes[r]);
        }
        {
            const float hxu = 0.5f * V.au[0], hyu = 0.5f * V.au[1], hxn = 0.5f * V.an[0], hyn = 0.5f * V.an[1];
            V.cdu[0] = -hxu - hyu; V.cdu[1] = hxu - hyu; V.cdu[2] = hyu - hxu; V.cdu[3] = hxu + hyu;
            V.cdn[0] = -hxn - hyn; V.cdn[1] = hxn - hyn; V.cdn[2] = hyn - hxn; V.cdn[3] = hxn + hyn;
            V.hzv = 0.5f * V.av[2];
            V.hzn = 0.5f * V.an[2];
        }
        V.o[0] = (float)o.x; V.o[1] = (float)o.y; V.o[2] = (float)o.z;
        V.eu[0] = (float)eu.x; V.eu[1] = (float)eu.y; V.eu[2] = (float)eu.z;
        V.ev[0] = (float)ev.x; V.ev[1] = (float)ev.y; V.ev[2] = (float)ev.z;
        V.nn[0] = (float)n.x; V.nn[1] = (float)n.y; V.nn[2] = (float)n.z;
        V.Ku = (float)(D / g->du);
        V.Cu = (float)(0.5 * (g->nu - 1) - u0 / g->du);
        V.Kv = (float)(D / g->dv);
        V.Cv = (float)(0.5 * (g->nv - 1) - h0 / g->dv);
        V.D = (float)D;
        V.main_y = std::fabs(cs.y) >= std::fabs(cs.x) ? 1 : 0;
        const double R = -dot(s, n);  // recon mode: source to rotation centre along n
        V.rc_R = (float)R;
        const double db = dbeta[v];
        V.rc_w = (float)(curved ? db : db * R * D);
        {  // ramp's response to a constant row, in FP64 (a small difference of large sums)
            const double st = curved ? g->du / D : g->du;
            double sum = 1.0 / (8.0 * st * st);
            for (int k = 1; k < g->nu; k += 2) {
                const double den = curved ? std::sin(k * st) : k * st;
                sum -= 1.0 / (M_PI * M_PI * den * den);
            }
            V.rc_c = (float)(st * sum);
        }

        // The volume must lie between source and detector; bound the
        // footprint extents (in cells) for the forward-gather search windows.
        double bmin = 1e300, bmax = -1e300, tu = 0, tv = 0, rmax = 0;
        for (int q = 0; q < 8; ++q) {
            const Vec3 X{X0.x + ((q & 1) ? (g->nx - 0.5) * g->dx : -0.5 * g->dx),
                         X0.y + ((q & 2) ? (g->ny - 0.5) * g->dy : -0.5 * g->dy),
                         X0.z + ((q & 4) ? (g->nz - 0.5) * g->dz : -0.5 * g->dz)};
            const Vec3 w = X - s;
            const double a = dot(w, eu), b = dot(w, n), cc = dot(w, ev);
            bmin = std::min(bmin, b);
            bmax = std::max(bmax, b);
            rmax = std::max(rmax, std::sqrt(a * a + b * b));
            if (b > 0) {
                tu = std::max(tu, std::fabs(a / b));
                tv = std::max(tv, std::fabs(cc / b));
            }
        }
        if (!(bmin > 0) || (!curved && !(bmax < D)) || (curved && !(rmax < D))) {
            delete g;
            return fail(CT_ERR_INVALID_ARG,
                        "view " + std::to_string(v) + ": the volume is not between the source and the detector");
        }
        auto bound = [&](double K, double alpha, double beta, double t) {
            const double den = bmin - beta;
            if (!(den > 0)) return 1e30;
            return 1.001 * K * (alpha + t * beta) / den + 1e-4;
        };
        const double hx = 0.5 * g->dx, hy = 0.5 * g->dy, hz = 0.5 * g->dz;
        V.m_sf_u = (float)bound(D / g->du, hx * std::fabs(eu.x) + hy * std::fabs(eu.y),
                                hx * std::fabs(n.x) + hy * std::fabs(n.y), tu);
        V.m_sf_v = (float)bound(D / g->dv, hz * std::fabs(ev.z), hz * std::fabs(n.z), tv);
        // SF-TT: the z faces at the transaxial corners (a 2D row lies inside the
        // axial plateau, so its factor is 1 and the bound does not matter)
        V.m_tt_v = two_d ? 0.25f
                         : (float)bound(D / g->dv, hx * std::fabs(ev.x) + hy * std::fabs(ev.y) + hz * std::fabs(ev.z),
                                        hx * std::fabs(n.x) + hy * std::fabs(n.y) + hz * std::fabs(n.z), tv);
        if (V.main_y)
            V.m_dd_u = (float)bound(D / g->du, hx * std::fabs(eu.x), hx * std::fabs(n.x), tu);
        else
            V.m_dd_u = (float)bound(D / g->du, hy * std::fabs(eu.y), hy * std::fabs(n.y), tu);
        if (V.m_sf_u > 1e6f || V.m_sf_v > 1e6f) {
            delete g;
            return fail(CT_ERR_INVALID_ARG, "view " + std::to_string(v) + ": voxels too close to the source");
        }
    }

    CtGrid &G = g->grid;
    G.nx = g->nx; G.ny = g->ny; G.nz = g->nz;
    G.nu = g->nu; G.nv = g->nv; G.nview = g->nview;
    G.dx = (float)g->dx; G.dy = (float)g->dy; G.dz = (float)g->dz;
    G.du = (float)g->du; G.dv = (float)g->dv;
    G.is2d = two_d ? 1 : 0;
    G.variant = d->kind == CT_NONCIRC3D ? ctp::GEO_NONCIRC_FLAT
                                        : (curved ? ctp::GEO_CIRC_CURVED : ctp::GEO_CIRC_FLAT);
    G.alpha = 1.f;
    G.beta = 0.f;
    G.max_m_sf_u = 0.f;
    G.max_m_dd_u = 0.f;
    G.max_m_sf_v = 0.f;
    G.max_m_tt_v = 0.f;
    for (const CtView &V : g->host_views) {
        G.max_m_sf_u = std::max(G.max_m_sf_u, V.m_sf_u);
        G.max_m_dd_u = std::max(G.max_m_dd_u, V.m_dd_u);
        G.max_m_sf_v = std::max(G.max_m_sf_v, V.m_sf_v);
        G.max_m_tt_v = std::max(G.max_m_tt_v, V.m_tt_v);
    }

    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(CT_ERR_CUDA, "no CUDA device");
    }
    const size_t bytes = sizeof(CtView) * g->host_views.size();
    cudaError_t e = cudaMalloc(&g->dev_views, bytes);
    if (e != cudaSuccess) {
        delete g;
        return fail(e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA,
                    std::string("geometry table allocation: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(g->dev_views, g->host_views.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->dev_views);
        delete g;
        return fail(CT_ERR_CUDA, std::string("geometry table upload: ") + cudaGetErrorString(e));
    }
    *out = g;
    return CT_OK;
}

ct_status ct_geometry_destroy(ct_geometry *g) {
    if (!g) return CT_OK;
    ct_status st = CT_OK;
    if (g->dev_views) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != g->device) cudaSetDevice(g->device);
        if (cudaFree(g->dev_views) != cudaSuccess) st = fail(CT_ERR_CUDA, "cudaFree of the geometry table failed");
        if (cur != g->device && cur >= 0) cudaSetDevice(cur);
    }
    delete g;
    return st;
}

ct_status ct_geometry_shape(const ct_geometry *g, int *nx, int *ny, int *nz, int *nu, int *nv, int *nview) {
    if (!g) return fail(CT_ERR_INVALID_ARG, "null geometry");
    if (nx) *nx = g->nx;
    if (ny) *ny = g->ny;
    if (nz) *nz = g->nz;
    if (nu) *nu = g->nu;
    if (nv) *nv = g->nv;
    if (nview) *nview = g->nview;
    return CT_OK;
}

static ct_status check_ptr(const void *p, const char *what) { return ctp::check_device_ptr(p, what); }

static ct_status project(int dir, const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t,
                         const void *in, ct_dtype out_t, void *out, int batch, float alpha, float beta,
                         void *stream) {
    if (!g) return fail(CT_ERR_INVALID_ARG, "null geometry");
    if (proj < CT_VOXEL || proj > CT_SF_TT) return fail(CT_ERR_INVALID_ARG, "unknown projector");
    if (mode != CT_MODE_PROJ && mode != CT_MODE_RECON) return fail(CT_ERR_INVALID_ARG, "unknown mode");
    if (mode == CT_MODE_RECON && (dir != 1 || (proj != CT_VOXEL && proj != CT_DD && proj != CT_SF)))
        return fail(CT_ERR_UNSUPPORTED, "recon mode is the FBP backprojection (ct_back) of CT_VOXEL, CT_DD, CT_SF");
    if (in_t < CT_F32 || in_t > CT_BF16 || out_t < CT_F32 || out_t > CT_BF16)
        return fail(CT_ERR_INVALID_ARG, "unknown dtype");
    if (!in || !out) return fail(CT_ERR_INVALID_ARG, "null data pointer");
    if (batch < 1) return fail(CT_ERR_INVALID_ARG, "batch must be >= 1");
    if ((proj == CT_SF || proj == CT_SF_TT) && std::fabs(g->dx - g->dy) > 1e-9 * g->dx)
        return fail(CT_ERR_UNSUPPORTED, "the SF amplitude needs square voxels (dx == dy)");
    if (proj == CT_SF_TT && g->grid.variant == ctp::GEO_CIRC_CURVED)
        return fail(CT_ERR_UNSUPPORTED, "SF-TT is provided for flat detectors");
    if (proj == CT_SF_TT && !ctp::nc_footprint_fits(g->grid, 2))
        return fail(CT_ERR_UNSUPPORTED, "SF-TT footprints wider than 8 cells or taller than 4 rows");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return fail(CT_ERR_INVALID_ARG, "the geometry's device is not the current device");
    const long long tiles =
        dir == 0 ? (long long)((g->nu + 31) / 32) * g->nview * batch
                 : (long long)((g->nx + 31) / 32) * ((g->nz + 7) / 8) * batch;
    if (tiles > 2147483647LL) return fail(CT_ERR_INVALID_ARG, "batch too large for one launch");
    ct_status st = check_ptr(in, "input");
    if (st != CT_OK) return st;
    st = check_ptr(out, "output");
    if (st != CT_OK) return st;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(CT_ERR_INVALID_ARG, "alpha and beta must be finite");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CtGrid G = g->grid;
    G.alpha = alpha;
    G.beta = beta;
    cudaError_t e;
    switch (mode == CT_MODE_RECON ? -1 - (int)proj : (int)proj) {
    case -1 - CT_VOXEL: e = ctp::launch_voxel_recon(G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case -1 - CT_DD: e = ctp::launch_recon_fp(1, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case -1 - CT_SF: e = ctp::launch_recon_fp(0, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case CT_VOXEL: e = ctp::launch_voxel(dir, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case CT_RAY: e = ctp::launch_ray(dir, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case CT_DD: e = ctp::launch_dd(dir, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    case CT_SF_TT: e = ctp::launch_sftt(dir, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    default: e = ctp::launch_sf(dir, G, g->dev_views, in_t, in, out_t, out, batch, s); break;
    }
    if (e == cudaErrorMemoryAllocation) return fail(CT_ERR_OOM, "workspace allocation failed");
    if (e == cudaErrorNotSupported)
        return fail(CT_ERR_UNSUPPORTED, "recon mode: non-circular footprints wider than 8 cells x 4 rows");
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return CT_OK;
}

ct_status ct_forward(const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t, const void *vol,
                     ct_dtype out_t, void *sino, int batch, void *cuda_stream) {
    return project(0, g, proj, mode, in_t, vol, out_t, sino, batch, 1.f, 0.f, cuda_stream);
}

ct_status ct_back(const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t, const void *sino,
                  ct_dtype out_t, void *vol, int batch, void *cuda_stream) {
    return project(1, g, proj, mode, in_t, sino, out_t, vol, batch, 1.f, 0.f, cuda_stream);
}

ct_status ct_forward_acc(const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t, const void *vol,
                         ct_dtype out_t, void *sino, int batch, float alpha, float beta, void *cuda_stream) {
    return project(0, g, proj, mode, in_t, vol, out_t, sino, batch, alpha, beta, cuda_stream);
}

ct_status ct_back_acc(const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t, const void *sino,
                      ct_dtype out_t, void *vol, int batch, float alpha, float beta, void *cuda_stream) {
    return project(1, g, proj, mode, in_t, sino, out_t, vol, batch, alpha, beta, cuda_stream);
}

// Pooled workspace of one projection call, by the same rules the launchers
// follow (k_sf.cu, k_nc_fwd.cu, k_nc_back.cu, k_ray.cu).
static size_t workspace_rule(int dir, const ct_geometry *g, ct_projector proj, ct_mode mode, ct_dtype in_t,
                             int batch) {
    const CtGrid &G = g->grid;
    const size_t vox = (size_t)g->nx * g->ny * g->nz * (size_t)batch;
    const size_t cells = (size_t)g->nview * g->nv * g->nu * (size_t)batch;
    const size_t isz = in_t == CT_F32 ? 4 : 2;
    const bool nc = G.variant == ctp::GEO_NONCIRC_FLAT;
    const bool zmajor = !G.is2d && g->nz % 4 == 0 && g->nz >= 8;  // the streaming forward's copy
    if (mode == CT_MODE_RECON) return 0;
    if (dir == 0) {
        switch (proj) {
        case CT_VOXEL: return !nc && zmajor ? vox * isz : 0;
        case CT_RAY: return 0;
        case CT_DD:
            if (nc) return ctp::nc_footprint_fits(G, 1) ? vox * isz : 0;
            return G.max_m_dd_u <= 3.5f && zmajor ? vox * isz : 0;
        case CT_SF:
            if (nc) return ctp::nc_footprint_fits(G, 0) ? vox * isz : 0;
            return G.max_m_sf_u <= 3.5f && zmajor ? vox * isz : 0;
        default:  // SF-TT: streaming forward in circular flat 3D geometry, footprint forward otherwise
            return ctp::sftt_circ_fits(G) ? (zmajor ? vox * isz : 0) : vox * isz;
        }
    }
    switch (proj) {
    case CT_RAY: return nc ? 0 : cells * 4;
    case CT_DD: return !nc || ctp::nc_footprint_fits(G, 1) ? cells * 4 : 0;
    case CT_SF_TT: return cells * 4;
    default: return 0;
    }
}

ct_status ct_workspace_bytes(const ct_geometry *g, ct_projector proj, ct_mode mode, int direction, ct_dtype in_t,
                             int batch, size_t *bytes) {
    if (!g || !bytes) return fail(CT_ERR_INVALID_ARG, "null geometry or output pointer");
    if (proj < CT_VOXEL || proj > CT_SF_TT) return fail(CT_ERR_INVALID_ARG, "unknown projector");
    if (mode != CT_MODE_PROJ && mode != CT_MODE_RECON) return fail(CT_ERR_INVALID_ARG, "unknown mode");
    if (direction != 0 && direction != 1) return fail(CT_ERR_INVALID_ARG, "direction must be 0 (forward) or 1 (back)");
    if (in_t < CT_F32 || in_t > CT_BF16) return fail(CT_ERR_INVALID_ARG, "unknown dtype");
    if (batch < 1) return fail(CT_ERR_INVALID_ARG, "batch must be >= 1");
    *bytes = workspace_rule(direction, g, proj, mode, in_t, batch);
    return CT_OK;
}

ct_status ct_workspace_limit(size_t bytes) {
    const cudaError_t e = ctp::workspace_set_limit(bytes);
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("workspace pool: ") + cudaGetErrorString(e));
    return CT_OK;
}

ct_status ct_workspace_usage(size_t *reserved, size_t *used_high, int reset_high) {
    const cudaError_t e = ctp::workspace_usage(reserved, used_high, reset_high);
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("workspace pool: ") + cudaGetErrorString(e));
    return CT_OK;
}

ct_status ct_ramp_filter(const ct_geometry *g, ct_dtype in_t, const void *sino, ct_dtype out_t, void *out, int batch,
                         void *cuda_stream) {
    if (!g) return fail(CT_ERR_INVALID_ARG, "null geometry");
    if (in_t < CT_F32 || in_t > CT_BF16 || out_t < CT_F32 || out_t > CT_BF16)
        return fail(CT_ERR_INVALID_ARG, "unknown dtype");
    if (!sino || !out) return fail(CT_ERR_INVALID_ARG, "null data pointer");
    if (batch < 1) return fail(CT_ERR_INVALID_ARG, "batch must be >= 1");
    if (sino == out && in_t != out_t) return fail(CT_ERR_INVALID_ARG, "an in-place filter keeps the type");
    if (g->nu > 16384) return fail(CT_ERR_UNSUPPORTED, "rows longer than 16384 cells");
    if ((long long)g->nv * g->nview * batch > 2147483647LL) return fail(CT_ERR_INVALID_ARG, "too many rows");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return fail(CT_ERR_INVALID_ARG, "the geometry's device is not the current device");
    ct_status st = check_ptr(sino, "input");
    if (st != CT_OK) return st;
    st = check_ptr(out, "output");
    if (st != CT_OK) return st;
    cudaError_t e = ctp::launch_ramp_filter(g->grid, g->dev_views, in_t, sino, out_t, out, batch,
                                            static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return CT_OK;
}

}  // extern "C"
