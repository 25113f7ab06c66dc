// ct_types.h -- per-view geometry records shared by the host set-up and the
// CUDA kernels.  Plain C++ (no CUDA headers) so both compilers see one layout.
#pragma once
#include <cstddef>
#include <cstdint>

namespace ctp {

// One record per view, computed in FP64 on the host and rounded once.
// Voxel index coordinates: X~ = (i, j, k, 1).  With w = X - s (voxel centre
// minus source, mm), the three detector-frame components of w are affine in
// X~:  w.e_u = au . X~,  w.e_v = av . X~,  w.n = an . X~.
// Fractional detector coordinates (cell a covers [a - 1/2, a + 1/2]):
//   flat:   fu = Ku (w.e_u)/(w.n) + Cu,        fv = Kv (w.e_v)/(w.n) + Cv
//   curved: fu = Ku atan2(w.e_u, w.n) + Cu,    fv = Kv (w.e_v)/rho + Cv,
//           rho = sqrt((w.e_u)^2 + (w.n)^2)
// with Ku = D/du, Kv = D/dv, Cu = (nu-1)/2 - u0/du, Cv = (nv-1)/2 - h0/dv and
// D = (c - s).n (flat) or the cylinder radius (curved).
struct alignas(16) CtView {
    float au[4];
    float av[4];
    float an[4];
    float o[4];       // w of voxel (0,0,0): first voxel centre minus source (mm)
    float eu[4];      // detector axis e_u (world), [3] unused
    float ev[4];      // detector axis e_v (world), [3] unused
    float nn[4];      // detector normal n = e_u x e_v (world), [3] unused
    float Ku, Cu, Kv, Cv;
    float D;          // (c - s).n, or the radius of a curved detector
    int main_y;       // slab axis of the view: 1 = y (|d_y| >= |d_x| of the central ray)
    float m_sf_u;     // bound on |fu(corner) - fu(centre)| over the volume (SF), cells
    float m_sf_v;     // bound on |fv(z +- dz/2) - fv(centre)| (SF and DD), rows
    float m_dd_u;     // bound on |fu(boundary point) - fu(centre)| (DD), cells
    float rc_w;       // recon mode: flat dbeta R D, curved dbeta (dbeta = the view's share of the gantry angle)
    float rc_R;       // recon mode: R = (O - s).n, the source's distance to the rotation centre O
    float rc_c;       // recon mode: step (h0 + 2 sum_{odd k < nu} h_k), the ramp's response to a constant row
    float m_tt_v;     // bound on the SF-TT axial knots' distance from fv(centre), rows
    // offsets of a voxel's four transaxial corners from its centre (corners
    // (-,-), (+,-), (-,+), (+,+) in (x, y)) along e_u and along n, and half
    // its height along e_v and n (mm; single precision, as the kernels use them)
    float cdu[4], cdn[4];
    float hzv, hzn;
    float pad;
};
static_assert(sizeof(CtView) == 52 * 4, "CtView layout");

enum GeoVariant { GEO_CIRC_FLAT = 0, GEO_CIRC_CURVED = 1, GEO_NONCIRC_FLAT = 2 };

// Sizes shared by all views.
struct CtGrid {
    int nx, ny, nz;
    int nu, nv, nview;
    float dx, dy, dz;
    float du, dv;
    int is2d;          // fan beam: single slice, unit slice thickness and row height
    int variant;       // GeoVariant
    float max_m_sf_u;  // largest per-view SF transaxial footprint bound (cells)
    float max_m_dd_u;  // largest per-view DD boundary bound (cells)
    float max_m_sf_v;  // largest per-view axial half-height bound (rows)
    float max_m_tt_v;  // largest per-view SF-TT axial bound (rows)
    float alpha, beta; // output epilogue: out = alpha * result + beta * out
};

}  // namespace ctp
