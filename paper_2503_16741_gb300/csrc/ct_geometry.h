// ct_geometry.h -- the library's geometry object behind the opaque
// ct_geometry handle of include/ctproj.h (host copy of the sizes and the
// per-view records, and their device copy).
#pragma once
#include <string>
#include <vector>

#include "../../include/ctproj.h"
#include "ct_types.h"

struct ct_geometry {
    int kind = 0, det = 0;
    int nx = 0, ny = 0, nz = 0, nu = 0, nv = 0, nview = 0;
    double dx = 0, dy = 0, dz = 0, du = 0, dv = 0;
    ctp::CtGrid grid{};
    std::vector<ctp::CtView> host_views;
    ctp::CtView *dev_views = nullptr;
    int device = -1;
};

namespace ctp {
// message returned by ct_last_error() on this thread
void set_last_error(const std::string &msg);
// CT_OK if p is device or managed memory, else CT_ERR_INVALID_ARG (message set)
ct_status check_device_ptr(const void *p, const char *what);
}  // namespace ctp
