// layout.cu -- FP64 host construction of the log-polar layout and of the device
// tables shared by all sessions with the same acuity model.
#include "layout.h"
#include "vafr_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

namespace vafr {

int Mapping::init(const vafr_acuity& a) {
    if (a.n_pivots < 2 || a.n_pivots > VAFR_MAX_PIVOTS) return -1;
    if (a.pivot_ecc_deg[0] != 0.0) return -1;
    for (int k = 0; k < a.n_pivots; ++k) {
        if (!std::isfinite(a.pivot_ecc_deg[k]) || !(a.pivot_cpd[k] > 0.0) || !std::isfinite(a.pivot_cpd[k]))
            return -1;
        if (k > 0 && !(a.pivot_ecc_deg[k] > a.pivot_ecc_deg[k - 1])) return -1;
    }
    if (!(a.e_max_deg > 0.0) || !(a.e_max_deg < 90.0)) return -1;
    aniso = a.anisotropic != 0;
    for (int k = 0; k < a.n_pivots; ++k) {
        if (aniso && !(a.pivot_delta[k] > 0.0 && std::isfinite(a.pivot_delta[k]))) return -1;
        delta[k] = aniso ? a.pivot_delta[k] : 1.0;
    }
    n_seg = a.n_pivots - 1;
    e_max = a.e_max_deg;
    U[0] = 0.0;
    for (int i = 0; i < n_seg; ++i) {
        E[i] = a.pivot_ecc_deg[i];
        const double w_lo = 1.0 / a.pivot_cpd[i], w_hi = 1.0 / a.pivot_cpd[i + 1];
        const double span = a.pivot_ecc_deg[i + 1] - E[i];
        m[i] = (w_hi - w_lo) / span;
        w[i] = w_lo - m[i] * E[i];
        U[i + 1] = U[i] + du(i, span);
    }
    E[n_seg] = a.pivot_ecc_deg[n_seg];
    // MAR must stay positive up to e_max (it is extrapolated past the last pivot)
    for (int i = 0; i < n_seg; ++i)
        if (!(m[i] * E[i] + w[i] > 0.0)) return -1;
    if (!(m[n_seg - 1] * e_max + w[n_seg - 1] > 0.0)) return -1;
    return 0;
}

double Mapping::du(int i, double de) const {
    const double om0 = m[i] * E[i] + w[i];
    if (m[i] == 0.0) return 2.0 * de / w[i];
    return 2.0 / m[i] * std::log1p(m[i] * de / om0);
}

int Mapping::seg_e(double e) const {
    int i = 0;
    while (i + 1 < n_seg && e >= E[i + 1]) ++i;
    return i;
}

double Mapping::u_of_e(double e) const {
    const int i = seg_e(e);
    return U[i] + du(i, e - E[i]);
}

double Mapping::e_of_u(double u) const {
    int i = 0;
    while (i + 1 < n_seg && u >= U[i + 1]) ++i;
    const double om0 = m[i] * E[i] + w[i];
    if (m[i] == 0.0) return E[i] + (u - U[i]) * w[i] / 2.0;
    return E[i] + std::expm1(m[i] * (u - U[i]) / 2.0) * om0 / m[i];
}

double Mapping::l_of_e(double e) const {
    const int i = seg_e(e);
    return 360.0 * std::sin(2.0 * e * M_PI / 180.0) / (m[i] * e + w[i]);
}

double Mapping::delta_of_e(double e) const {
    if (!aniso) return 1.0;
    if (e >= E[n_seg]) return delta[n_seg];
    const int i = seg_e(e);
    return delta[i] + (e - E[i]) / (E[i + 1] - E[i]) * (delta[i + 1] - delta[i]);
}

double Mapping::du_de(double e) const {
    const int i = seg_e(e);
    return 2.0 / (m[i] * e + w[i]);
}

LayoutTables::~LayoutTables() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    cudaFree(d_tan_e);
    cudaFree(d_col);
    cudaFree(d_col_pair);
    cudaFree(d_u_tab);
    cudaFree(d_work);
    cudaSetDevice(cur);
}

namespace {

// Cubic Hermite pieces of u(z) - 1/2 (the bilinear filter's column
// coordinate), z = tan(e), on kUTable uniform intervals of [0, tan(e_max)],
// from the exact u and du/dz = du/de (180/pi) / (1 + z^2), plus one constant
// entry u(e_max) - 1/2 for the clamp.
void build_u_table(const Mapping& mp, std::vector<float4>& tab, double& inv_h) {
    const int N = kUTable;
    const double z_max = std::tan(mp.e_max * M_PI / 180.0);
    const double h = z_max / N;
    std::vector<double> p(N + 1), d(N + 1);
    for (int k = 0; k <= N; ++k) {
        const double z = k == N ? z_max : k * h;
        const double e = k == N ? mp.e_max : std::atan(z) * 180.0 / M_PI;
        p[k] = mp.u_of_e(e);
        d[k] = mp.du_de(e) * (180.0 / M_PI) / (1.0 + z * z) * h;
    }
    tab.resize(N + 1);
    for (int k = 0; k < N; ++k) {
        const double c2 = 3.0 * (p[k + 1] - p[k]) - 2.0 * d[k] - d[k + 1];
        const double c3 = 2.0 * (p[k] - p[k + 1]) + d[k] + d[k + 1];
        tab[k] = make_float4((float)(p[k] - 0.5), (float)d[k], (float)c2, (float)c3);
    }
    tab[N] = make_float4((float)(p[N] - 0.5), 0.0f, 0.0f, 0.0f);   // z >= tan(e_max): u(e_max)
    inv_h = N / z_max;
}

int32_t float_bits(int32_t n) {
    const float f = (float)n;
    int32_t b;
    std::memcpy(&b, &f, sizeof(b));
    return b;
}

// Position of cell (x, y) of a 2^16 x 2^16 grid along the Hilbert curve:
// from the coarsest level down, each level adds its quadrant's rank (0-3 in
// curve order) and turns the remaining coordinates into that quadrant's
// frame (a transpose, mirrored for the last quadrant).
uint32_t hilbert16(uint32_t x, uint32_t y) {
    uint32_t d = 0;
    for (uint32_t s = 1u << 15; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = (s - 1) - (x & (s - 1)) + (x & ~(s - 1));
                y = (s - 1) - (y & (s - 1)) + (y & ~(s - 1));
            }
            const uint32_t t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// Processing order of the LP texels: Hilbert order of each texel's screen
// direction relative to the gaze, (tan e_c cos phi_j, tan e_c sin phi_j), so the
// 32 rays a warp takes are spatial neighbours (the curve has no long jumps
// between consecutive cells).  This direction depends on the acuity model
// only, never on the display size or the gaze.
void build_work_order(const LayoutTables& L, std::vector<int2>& work) {
    const double X = std::tan(L.map.e_max * M_PI / 180.0) * 1.0001;
    // (Hilbert key, slot, column); the slot breaks ties, so the order is a function
    std::vector<std::pair<uint32_t, int2>> key;
    key.reserve(L.n_texels);
    for (int c = 0; c < L.n_cols; ++c) {
        const double te = std::tan(L.e_col[c] * M_PI / 180.0);
        for (int32_t j = 0; j < L.n_col[c]; ++j) {
            const double ph = 2.0 * M_PI * (j + 0.5) / L.n_col[c];
            const double x = te * std::cos(ph), y = te * std::sin(ph);
            const uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, (x + X) / (2 * X) * 65535.0));
            const uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, (y + X) / (2 * X) * 65535.0));
            key.push_back({hilbert16(qx, qy), make_int2((int)(L.off_col[c] + j), c)});
        }
    }
    std::sort(key.begin(), key.end(), [](const std::pair<uint32_t, int2>& a, const std::pair<uint32_t, int2>& b) {
        return a.first != b.first ? a.first < b.first : a.second.x < b.second.x;
    });
    work.resize(L.n_texels);
    for (int64_t w = 0; w < L.n_texels; ++w) work[w] = key[w].second;
}

int build(const vafr_acuity& acuity, LayoutTables& L, std::string* err) {
    if (L.map.init(acuity) != 0) {
        *err = "bad acuity pivots (need E_0 = 0, increasing pivots, f > 0, 0 < e_max < 90, MAR > 0, "
               "delta > 0 when anisotropic)";
        return VAFR_ERR_INVALID_ARG;
    }
    // Column c occupies slots [off_c - 1, off_c + n_c]: its n_c texels plus a
    // guard slot on each side holding a copy of the texel across the angular
    // wrap (texel n_c - 1 before, texel 0 after), so a bilinear row pair is
    // always two adjacent slots.
    const double u_max = L.map.u_of_e(L.map.e_max);
    int64_t acc = 0, slots = 0;
    for (int c = 0; (double)c + 0.5 < u_max; ++c) {
        const double e = L.map.e_of_u((double)c + 0.5);
        int32_t nc = (int32_t)std::floor(L.map.delta_of_e(e) * L.map.l_of_e(e) + 0.5);
        if (nc < 1) nc = 1;
        L.e_col.push_back(e);
        L.n_col.push_back(nc);
        L.off_col.push_back(slots + 1);
        acc += nc;
        slots += nc + 2;
        if (slots > (1ll << 28) || L.e_col.size() > (1u << 20)) {
            *err = "LP layout too large";
            return VAFR_ERR_INVALID_ARG;
        }
    }
    L.n_cols = (int)L.e_col.size();
    L.n_texels = acc;
    L.n_slots = slots;
    if (L.n_cols == 0) {
        *err = "empty LP layout";
        return VAFR_ERR_INVALID_ARG;
    }
    std::vector<float> tan_e(L.n_cols);
    std::vector<int2> col(L.n_cols);
    // entry 0 pairs column 0 with itself (for u - 1/2 < 0), entry c + 1 pairs c
    // with min(c + 1, C - 1); the device pointer handed to kernels is entry 1.
    // Counts are stored as FP32 bit patterns: the filter only uses n_c as a float.
    std::vector<int4> col_pair(L.n_cols + 1);
    for (int c = 0; c < L.n_cols; ++c) {
        tan_e[c] = (float)std::tan(L.e_col[c] * M_PI / 180.0);
        col[c] = make_int2((int)L.off_col[c], L.n_col[c]);
    }
    for (int c = 0; c < L.n_cols; ++c) {
        const int c1 = c + 1 < L.n_cols ? c + 1 : c;
        col_pair[c + 1] = make_int4(col[c].x, float_bits(col[c].y), col[c1].x, float_bits(col[c1].y));
    }
    col_pair[0] = make_int4(col[0].x, float_bits(col[0].y), col[0].x, float_bits(col[0].y));
    std::vector<float4> u_tab;
    build_u_table(L.map, u_tab, L.u_inv_h);
    std::vector<int2> work;
    build_work_order(L, work);
    cudaError_t e = cudaSuccess;
    auto up = [&](auto** dst, const auto& src) {
        if (e != cudaSuccess) return;
        const size_t bytes = sizeof(src[0]) * src.size();
        e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), bytes, cudaMemcpyHostToDevice);
    };
    up(&L.d_tan_e, tan_e);
    up(&L.d_col, col);
    up(&L.d_col_pair, col_pair);
    up(&L.d_u_tab, u_tab);
    up(&L.d_work, work);
    if (e != cudaSuccess) {
        *err = std::string("layout tables: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? VAFR_ERR_OOM : VAFR_ERR_CUDA;
    }
    return VAFR_OK;
}

std::mutex g_mu;
std::map<std::string, std::weak_ptr<const LayoutTables>> g_cache;

}  // namespace

int get_layout(const vafr_acuity& acuity, std::shared_ptr<const LayoutTables>* out, std::string* err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *err = "cudaGetDevice failed";
        return VAFR_ERR_CUDA;
    }
    // key: device + the acuity model's defining values (padding bytes excluded)
    std::string key(reinterpret_cast<const char*>(&dev), sizeof(dev));
    key.append(reinterpret_cast<const char*>(&acuity.n_pivots), sizeof(acuity.n_pivots));
    const int np = acuity.n_pivots > 0 && acuity.n_pivots <= VAFR_MAX_PIVOTS ? acuity.n_pivots : 0;
    key.append(reinterpret_cast<const char*>(acuity.pivot_ecc_deg), sizeof(double) * np);
    key.append(reinterpret_cast<const char*>(acuity.pivot_cpd), sizeof(double) * np);
    key.append(reinterpret_cast<const char*>(&acuity.e_max_deg), sizeof(double));
    const int32_t aniso = acuity.anisotropic != 0;
    key.append(reinterpret_cast<const char*>(&aniso), sizeof(aniso));
    if (aniso) key.append(reinterpret_cast<const char*>(acuity.pivot_delta), sizeof(double) * np);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        if (auto sp = it->second.lock()) {
            *out = sp;
            return VAFR_OK;
        }
    }
    auto L = std::make_shared<LayoutTables>();
    L->device = dev;
    const int rc = build(acuity, *L, err);
    if (rc != VAFR_OK) return rc;
    g_cache[key] = L;
    *out = L;
    return VAFR_OK;
}

}  // namespace vafr
