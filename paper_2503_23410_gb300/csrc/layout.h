// layout.h -- host side of the log-polar layout: the FP64 acuity mapping and the
// per-acuity device tables (shared by every session with the same pivots).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/vafr.h"

namespace vafr {

// The segmented mapping (Sec. 3.3, Eq. 12) in FP64.  MAR omega = 1/f is
// piecewise linear through the pivots (E_k, 1/f_k) (Eq. 2 per segment); on
// segment i
//   u(e) = U_i + (2/m_i) ln(1 + m_i (e - E_i) / omega(E_i))      (Eq. 5 / 12)
// with U_0 = 0 and U_i making u continuous (the integration constants),
//   e(u) its inverse (Eq. 10), l(e) = 360 sin(2e) / omega(e) (Eqs. 8-9),
//   du/de = 2 / omega(e) (Eq. 4).  Flat segments (m_i = 0) use the limit.
// Anisotropy (Sec. 9, Eq. 19): Delta(e) piecewise linear through the pivots'
// deltas, constant past the last pivot; 1 for an isotropic model.
struct Mapping {
    int n_seg = 0;
    double E[VAFR_MAX_PIVOTS], m[VAFR_MAX_PIVOTS], w[VAFR_MAX_PIVOTS], U[VAFR_MAX_PIVOTS + 1];
    double e_max = 60.0;
    bool aniso = false;
    double delta[VAFR_MAX_PIVOTS];

    int init(const vafr_acuity& a);
    double du(int i, double de) const;
    int seg_e(double e) const;
    double u_of_e(double e) const;
    double e_of_u(double u) const;
    double l_of_e(double e) const;
    double delta_of_e(double e) const;
    double du_de(double e) const;
};

// Discrete layout (Sec. 3.2.2) and the device tables the kernels read.  The
// layout depends only on the acuity model, never on the display or the gaze.
struct LayoutTables {
    int device = 0;
    Mapping map;
    int n_cols = 0;
    int64_t n_texels = 0;           // sum of n_c: rays per eye
    int64_t n_slots = 0;            // LP buffer length: sum of (n_c + 2)
    std::vector<double> e_col;      // eccentricity of column centres u = c + 0.5
    std::vector<int32_t> n_col;     // texels per column
    std::vector<int64_t> off_col;   // slot of texel (c, 0); slots off - 1 and off + n_c are guards
    float* d_tan_e = nullptr;       // [C]
    int2* d_col = nullptr;          // [C] (slot of texel 0, count)
    int4* d_col_pair = nullptr;     // [C + 1]: entry c + 1 = (slot of texel 0, FP32 bits of the
                                    // count) of c and of min(c + 1, C - 1); entry 0 = column 0 twice
    float4* d_u_tab = nullptr;      // cubic pieces of u(z), z = tan(e)
    double u_inv_h = 0.0;
    int2* d_work = nullptr;         // [n_texels] (slot, column) in screen-space Morton order
    ~LayoutTables();
};

// Returns the tables of `acuity` on the current device, building them on first
// use; 0 on success, a VAFR_ERR_* code (with `err` filled) otherwise.
int get_layout(const vafr_acuity& acuity, std::shared_ptr<const LayoutTables>* out, std::string* err);

}  // namespace vafr
