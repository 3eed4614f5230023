// api.cu — host side of the C ABI declared in include/laueot.h: handle,
// workspace, argument validation and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "api_internal.h"

using namespace laue;

// ------------------------------------------------------------- helpers

int laue_fail(laue_handle* h, int code, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int laue_cuda_check(laue_handle* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LAUE_OK;
    return laue_fail(h, LAUE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

GeomDev laue_geom_dev(const LaueGeometry& g) {
    GeomDev d{};
    for (int a = 0; a < 3; ++a) d.e[a] = g.beam[a];
    d.lam_min = g.lam_min;
    d.lam_max = g.lam_max;
    d.D = g.D;
    d.n_det = g.n_det;
    for (int k = 0; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) {
            d.ctr[k][a] = g.det_centre[k][a];
            d.nrm[k][a] = g.det_normal[k][a];
        }
        d.half[k] = g.det_half[k];
        d.Dd[k] = g.det_D[k] > 0.0f ? g.det_D[k] : g.D;
        // in-plane axes a1 = (y x n)/|y x n| (x when n is along y), a2 = n x a1
        double nx = g.det_normal[k][0], ny = g.det_normal[k][1], nz = g.det_normal[k][2];
        double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
        if (nn > 0.0) {
            nx /= nn;
            ny /= nn;
            nz /= nn;
        }
        double a1[3] = {nz, 0.0, -nx};
        double l1 = std::sqrt(a1[0] * a1[0] + a1[2] * a1[2]);
        if (l1 < 1e-12) {
            a1[0] = 1.0;
            a1[2] = 0.0;
        } else {
            a1[0] /= l1;
            a1[2] /= l1;
        }
        double a2[3] = {ny * a1[2] - nz * a1[1], nz * a1[0] - nx * a1[2], nx * a1[1] - ny * a1[0]};
        for (int a = 0; a < 3; ++a) {
            d.ax1[k][a] = (float)a1[a];
            d.ax2[k][a] = (float)a2[a];
        }
    }
    return d;
}

int laue_check_geom(laue_handle* h, const LaueGeometry* g) {
    if (!g) return laue_fail(h, LAUE_ERR_INVALID_ARG, "geometry is NULL");
    if (g->n_det < 1 || g->n_det > 4) return laue_fail(h, LAUE_ERR_INVALID_ARG, "n_det must be 1..4");
    if (!(g->lam_min > 0.0f) || !(g->lam_max >= g->lam_min))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "wavelength band must satisfy 0 < lam_min <= lam_max");
    if (!(g->D > 0.0f)) return laue_fail(h, LAUE_ERR_INVALID_ARG, "D must be positive");
    for (int k = 0; k < g->n_det; ++k) {
        if (!(g->det_half[k] > 0.0f)) return laue_fail(h, LAUE_ERR_INVALID_ARG, "detector half size must be > 0");
        const float* n = g->det_normal[k];
        if (!(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] > 0.0f))
            return laue_fail(h, LAUE_ERR_INVALID_ARG, "detector normal must be nonzero");
        if (!(g->det_D[k] <= 0.0f || g->det_D[k] > 0.0f))
            return laue_fail(h, LAUE_ERR_INVALID_ARG, "detector cost length must be a number");
    }
    return LAUE_OK;
}

int laue_check_obs(laue_handle* h, const LaueObsSpots* o) {
    if (!o) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed spots are NULL");
    if (o->T < 1 || o->n < 0) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed spots: T >= 1 and n >= 0");
    if (!o->I_off) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed spots: I_off is NULL");
    if (o->n > 0 && (!o->p || !aligned16(o->p)))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed spots: p must be a 16-byte aligned device array");
    return LAUE_OK;
}

int laue_check_model(laue_handle* h, const LaueModelSpots* m) {
    if (!m) return laue_fail(h, LAUE_ERR_INVALID_ARG, "model spots are NULL");
    if (m->T < 1 || m->n < 0 || m->n > m->capacity)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "model spots: T >= 1 and 0 <= n <= capacity");
    if (!m->J_off) return laue_fail(h, LAUE_ERR_INVALID_ARG, "model spots: J_off is NULL");
    if (m->n > 0) {
        if (!m->grain || !m->plane || !m->angle || !m->ray || !m->center || !m->spot)
            return laue_fail(h, LAUE_ERR_INVALID_ARG, "model spots: a label or vector array is NULL");
        if (!aligned16(m->ray) || !aligned16(m->center) || !aligned16(m->spot))
            return laue_fail(h, LAUE_ERR_INVALID_ARG, "model spots: vector arrays must be 16-byte aligned");
    }
    return LAUE_OK;
}

int laue_need_ws(laue_handle* h, const LaueProblemDims& d, Layout* L) {
    *L = make_layout(d, h->sm_count);
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set (laue_set_workspace)");
    if (L->total > h->ws_bytes)
        return laue_fail(h, LAUE_ERR_WORKSPACE, "workspace too small: need %zu bytes, have %zu", L->total,
                         h->ws_bytes);
    return LAUE_OK;
}

// ------------------------------------------------------------- handle

extern "C" int laue_create(laue_handle** h, int device) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    *h = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LAUE_ERR_CUDA;
    laue_handle* H = (laue_handle*)calloc(1, sizeof(laue_handle));
    if (!H) return LAUE_ERR_INVALID_ARG;
    H->device = device;
    if (cudaDeviceGetAttribute(&H->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        free(H);
        return LAUE_ERR_CUDA;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    if (sinkhorn_occupancy(H->row_occ, H->col_occ) != 0)
        for (int v = 0; v < kSkVariants; ++v) H->row_occ[v] = H->col_occ[v] = 1;
    cudaSetDevice(prev);
    H->row_variant = H->col_variant = kSkDefaultVariant;
    H->skip = 1;
    H->err[0] = 0;
    *h = H;
    return LAUE_OK;
}

extern "C" int laue_destroy(laue_handle* h) {
    free(h);
    return LAUE_OK;
}

extern "C" const char* laue_last_error(const laue_handle* h) { return h ? h->err : "null handle"; }

extern "C" int laue_workspace_size(laue_handle* h, const LaueProblemDims* dims, size_t* bytes) {
    if (!h || !dims || !bytes) return laue_fail(h, LAUE_ERR_INVALID_ARG, "null argument");
    if (dims->T < 0 || dims->n_obs < 0 || dims->n_model < 0 || dims->n_grains < 0 || dims->n_planes < 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "negative dimension");
    *bytes = make_layout(*dims, h->sm_count).total;
    return LAUE_OK;
}

extern "C" int laue_set_workspace(laue_handle* h, void* dev_ptr, size_t bytes, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (dev_ptr && ((uintptr_t)dev_ptr & 255u))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (dev_ptr && bytes < kCtrlBytes) return laue_fail(h, LAUE_ERR_WORKSPACE, "workspace smaller than 4 KB");
    h->ws = dev_ptr;
    h->ws_bytes = dev_ptr ? bytes : 0;
    if (dev_ptr)
        return laue_cuda_check(h, cudaMemsetAsync(dev_ptr, 0, kCtrlBytes, (cudaStream_t)stream),
                               "clearing workspace control block");
    return LAUE_OK;
}

extern "C" int laue_device_status(laue_handle* h, void* stream, int* status_host) {
    if (!h || !status_host) return laue_fail(h, LAUE_ERR_INVALID_ARG, "null argument");
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    int rc = laue_cuda_check(h, cudaMemcpyAsync(&v, h->ws, sizeof(int), cudaMemcpyDeviceToHost, s),
                             "reading status");
    if (rc) return rc;
    rc = laue_cuda_check(h, cudaStreamSynchronize(s), "synchronising stream");
    if (rc) return rc;
    *status_host = v;
    return laue_cuda_check(h, cudaMemsetAsync(h->ws, 0, sizeof(int), s), "clearing status");
}

// ------------------------------------------------------------- host helper

namespace {
struct Refl {
    int g0[3];
    int n2, nh;
    double w[3], d0;
};
int gcd_i(int a, int b) {
    a = std::abs(a);
    b = std::abs(b);
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}
bool allowed(int h, int k, int l, int centering) {
    if (h == 0 && k == 0 && l == 0) return false;
    auto par = [](int v) { return ((v % 2) + 2) % 2; };
    if (centering == 1) return par(h + k + l) == 0;
    if (centering == 2) return par(h) == par(k) && par(k) == par(l);
    return true;
}
}  // namespace

extern "C" int laue_reflections(double a, int hmax, int centering, int cap, float* w_d0_host,
                                int* nharm_host, int* hkl0_host, int* M) {
    if (!M || hmax < 1 || hmax > 64 || !(a > 0.0) || centering < 0 || centering > 2 || cap < 0)
        return LAUE_ERR_INVALID_ARG;
    std::vector<Refl> list;
    for (int h = -hmax; h <= hmax; ++h)
        for (int k = -hmax; k <= hmax; ++k)
            for (int l = -hmax; l <= hmax; ++l) {
                if ((h == 0 && k == 0 && l == 0) || gcd_i(gcd_i(h, k), l) != 1) continue;
                int first = h != 0 ? h : (k != 0 ? k : l);
                if (first < 0) continue;  // one direction per Friedel pair
                int pmax = std::max(std::abs(h), std::max(std::abs(k), std::abs(l)));
                std::vector<int> mult;
                for (int m = 1; m * pmax <= hmax; ++m)
                    if (allowed(m * h, m * k, m * l, centering)) mult.push_back(m);
                if (mult.empty()) continue;
                for (size_t q = 0; q < mult.size(); ++q)
                    if (mult[q] != (int)(q + 1) * mult[0]) return LAUE_ERR_INVALID_ARG;
                Refl R;
                R.g0[0] = mult[0] * h;
                R.g0[1] = mult[0] * k;
                R.g0[2] = mult[0] * l;
                R.n2 = R.g0[0] * R.g0[0] + R.g0[1] * R.g0[1] + R.g0[2] * R.g0[2];
                R.nh = (int)mult.size();
                double pn = std::sqrt((double)(h * h + k * k + l * l));
                R.w[0] = h / pn;
                R.w[1] = k / pn;
                R.w[2] = l / pn;
                R.d0 = a / std::sqrt((double)R.n2);
                list.push_back(R);
            }
    std::sort(list.begin(), list.end(), [](const Refl& x, const Refl& y) {
        if (x.n2 != y.n2) return x.n2 < y.n2;
        for (int q = 0; q < 3; ++q)
            if (x.g0[q] != y.g0[q]) return x.g0[q] > y.g0[q];
        return false;
    });
    *M = (int)list.size();
    for (int m = 0; m < (int)list.size() && m < cap; ++m) {
        if (w_d0_host) {
            for (int q = 0; q < 3; ++q) w_d0_host[4 * m + q] = (float)list[m].w[q];
            w_d0_host[4 * m + 3] = (float)list[m].d0;
        }
        if (nharm_host) nharm_host[m] = list[m].nh;
        if (hkl0_host)
            for (int q = 0; q < 3; ++q) hkl0_host[3 * m + q] = list[m].g0[q];
    }
    return (int)list.size() > cap ? LAUE_ERR_CAPACITY : LAUE_OK;
}

extern "C" int laue_reciprocal_basis(double a, double b, double c, double alpha_deg, double beta_deg,
                                     double gamma_deg, double* B_host) {
    if (!B_host || !(a > 0.0) || !(b > 0.0) || !(c > 0.0) || !(alpha_deg > 0.0 && alpha_deg < 180.0) ||
        !(beta_deg > 0.0 && beta_deg < 180.0) || !(gamma_deg > 0.0 && gamma_deg < 180.0))
        return LAUE_ERR_INVALID_ARG;
    const double r = 3.14159265358979323846 / 180.0;
    double ca = std::cos(alpha_deg * r), cb = std::cos(beta_deg * r), cg = std::cos(gamma_deg * r);
    double sg = std::sin(gamma_deg * r);
    // direct basis: a1 along x, a2 in the xy plane, a3 completing it
    double a1[3] = {a, 0.0, 0.0}, a2[3] = {b * cg, b * sg, 0.0};
    double z1 = c * cb, z2 = c * (ca - cb * cg) / sg, zz = c * c - z1 * z1 - z2 * z2;
    if (!(zz > 0.0)) return LAUE_ERR_INVALID_ARG;  // the angles do not close a cell
    double a3[3] = {z1, z2, std::sqrt(zz)};
    auto cross = [](const double* u, const double* v, double* o) {
        o[0] = u[1] * v[2] - u[2] * v[1];
        o[1] = u[2] * v[0] - u[0] * v[2];
        o[2] = u[0] * v[1] - u[1] * v[0];
    };
    double c23[3], c31[3], c12[3];
    cross(a2, a3, c23);
    cross(a3, a1, c31);
    cross(a1, a2, c12);
    double V = a1[0] * c23[0] + a1[1] * c23[1] + a1[2] * c23[2];
    for (int i = 0; i < 3; ++i) {  // columns b1 = a2 x a3 / V, b2 = a3 x a1 / V, b3 = a1 x a2 / V
        B_host[3 * i + 0] = c23[i] / V;
        B_host[3 * i + 1] = c31[i] / V;
        B_host[3 * i + 2] = c12[i] / V;
    }
    return LAUE_OK;
}

extern "C" int laue_reflections_hkl(const double* B_host, const int* hkl_host, int n, int cap, float* w_d0_host,
                                    int* nharm_host, int* hkl0_host, int* M) {
    if (!M || !B_host || n < 0 || (n > 0 && !hkl_host) || cap < 0) return LAUE_ERR_INVALID_ARG;
    // every listed reflection on its line through the origin: primitive vector
    // (first nonzero index positive) and multiplier
    struct Item {
        int p[3];
        int m;
    };
    std::vector<Item> items;
    for (int q = 0; q < n; ++q) {
        int h = hkl_host[3 * q], k = hkl_host[3 * q + 1], l = hkl_host[3 * q + 2];
        if (h == 0 && k == 0 && l == 0) continue;
        int g = gcd_i(gcd_i(h, k), l);
        Item it{{h / g, k / g, l / g}, g};
        int first = it.p[0] != 0 ? it.p[0] : (it.p[1] != 0 ? it.p[1] : it.p[2]);
        if (first < 0)
            for (int a = 0; a < 3; ++a) it.p[a] = -it.p[a];
        items.push_back(it);
    }
    std::sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        for (int a = 0; a < 3; ++a)
            if (x.p[a] != y.p[a]) return x.p[a] < y.p[a];
        return x.m < y.m;
    });
    struct Ent {
        int g0[3];
        double len2, w[3], d0;
        int nh;
    };
    std::vector<Ent> out;
    for (size_t s = 0; s < items.size();) {
        size_t e = s;
        std::vector<int> mult;
        while (e < items.size() && items[e].p[0] == items[s].p[0] && items[e].p[1] == items[s].p[1] &&
               items[e].p[2] == items[s].p[2]) {
            if (mult.empty() || mult.back() != items[e].m) mult.push_back(items[e].m);
            ++e;
        }
        for (size_t q = 0; q < mult.size(); ++q)  // harmonics: m0, 2 m0, ..., nh m0
            if (mult[q] != (int)(q + 1) * mult[0]) return LAUE_ERR_INVALID_ARG;
        Ent E;
        for (int a = 0; a < 3; ++a) E.g0[a] = mult[0] * items[s].p[a];
        double g[3];
        for (int a = 0; a < 3; ++a)
            g[a] = B_host[3 * a] * E.g0[0] + B_host[3 * a + 1] * E.g0[1] + B_host[3 * a + 2] * E.g0[2];
        E.len2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        if (!(E.len2 > 0.0)) return LAUE_ERR_INVALID_ARG;
        double len = std::sqrt(E.len2);
        for (int a = 0; a < 3; ++a) E.w[a] = g[a] / len;
        E.d0 = 1.0 / len;
        E.nh = (int)mult.size();
        out.push_back(E);
        s = e;
    }
    std::sort(out.begin(), out.end(), [](const Ent& x, const Ent& y) {
        double tol = 1e-9 * std::max(x.len2, y.len2);
        if (std::fabs(x.len2 - y.len2) > tol) return x.len2 < y.len2;
        for (int q = 0; q < 3; ++q)
            if (x.g0[q] != y.g0[q]) return x.g0[q] > y.g0[q];
        return false;
    });
    *M = (int)out.size();
    for (int m = 0; m < (int)out.size() && m < cap; ++m) {
        if (w_d0_host) {
            for (int q = 0; q < 3; ++q) w_d0_host[4 * m + q] = (float)out[m].w[q];
            w_d0_host[4 * m + 3] = (float)out[m].d0;
        }
        if (nharm_host) nharm_host[m] = out[m].nh;
        if (hkl0_host)
            for (int q = 0; q < 3; ++q) hkl0_host[3 * m + q] = out[m].g0[q];
    }
    return (int)out.size() > cap ? LAUE_ERR_CAPACITY : LAUE_OK;
}

// ------------------------------------------------------------- forward

extern "C" int laue_forward(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                            const float* R, const float* x, int N, const float* omega, int T,
                            LaueModelSpots* out, int* total_host, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc = laue_check_geom(h, geom);
    if (rc) return rc;
    if (!lat || lat->M < 0 || (lat->M > 0 && (!lat->w_d0 || !lat->nharm || !aligned16(lat->w_d0))))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "lattice: M >= 0 and 16-byte aligned w_d0");
    if (N < 0 || T < 1 || !omega || (N > 0 && (!R || !x)) || !out || !total_host)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "forward: bad N, T or NULL array");
    if (out->T != T || !out->J_off || out->capacity < 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "forward: output list must have T = %d and J_off", T);
    if (out->capacity > 0 && (!out->grain || !out->plane || !out->angle || !out->ray || !out->center ||
                              !out->spot || !aligned16(out->ray) || !aligned16(out->center) ||
                              !aligned16(out->spot)))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "forward: output arrays NULL or misaligned");
    LaueProblemDims d{T, 0, 0, N, lat->M, 0, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    char* ws = (char*)h->ws;
    cudaStream_t s = (cudaStream_t)stream;
    FwdArgs a{};
    a.G = laue_geom_dev(*geom);
    a.R = R;
    a.x = x;
    a.omega = omega;
    a.w_d0 = (const float4*)lat->w_d0;
    a.nharm = lat->nharm;
    a.N = N;
    a.M = lat->M;
    a.T = T;
    a.n_rays = (long long)T * N * lat->M;
    a.n_blocks = (int)((a.n_rays + kFwdBlock - 1) / kFwdBlock);
    a.capacity = out->capacity;
    a.blocks = (int*)(ws + L.fwd_blocks);
    a.ctrl = (int*)(ws + L.ctrl);
    a.J_off = out->J_off;
    a.grain = out->grain;
    a.plane = out->plane;
    a.angle = out->angle;
    a.ray = (float4*)out->ray;
    a.center = (float4*)out->center;
    a.spot = (float4*)out->spot;
    if ((rc = laue_cuda_check(h, cudaMemsetAsync(out->J_off, 0, sizeof(int) * (T + 1), s), "clearing J_off")))
        return rc;
    if ((rc = laue_cuda_check(h, launch_forward(a, s), "forward launch"))) return rc;
    int total = 0;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(&total, a.ctrl + CTRL_FWD_TOTAL, sizeof(int),
                                                 cudaMemcpyDeviceToHost, s),
                              "reading spot count")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "forward synchronise"))) return rc;
    *total_host = total;
    out->n = std::min(total, out->capacity);
    if (total > out->capacity)
        return laue_fail(h, LAUE_ERR_CAPACITY, "forward: %d visible spots exceed capacity %d", total,
                         out->capacity);
    return LAUE_OK;
}

extern "C" int laue_refresh(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const float* R,
                            const float* x, const float* omega, LaueModelSpots* model, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc = laue_check_geom(h, geom);
    if (rc) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (!lat || (lat->M > 0 && (!lat->w_d0 || !lat->nharm)) || !R || !x || !omega)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "refresh: NULL array");
    RefreshArgs a{};
    a.G = laue_geom_dev(*geom);
    a.R = R;
    a.x = x;
    a.omega = omega;
    a.w_d0 = (const float4*)lat->w_d0;
    a.nharm = lat->nharm;
    a.n = model->n;
    a.grain = model->grain;
    a.plane = model->plane;
    a.angle = model->angle;
    a.ray = (float4*)model->ray;
    a.center = (float4*)model->center;
    a.spot = (float4*)model->spot;
    return laue_cuda_check(h, launch_refresh(a, (cudaStream_t)stream), "refresh launch");
}

// ------------------------------------------------------------- Sinkhorn

int laue_fill_sk(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs, const LaueModelSpots* model,
                 const LaueOTParams* prm, const Layout& L, SkArgs* out, SkLaunch* lc) {
    char* ws = (char*)h->ws;
    SkArgs a{};
    a.T = obs->T;
    a.n_obs = obs->n;
    a.n_model = model->n;
    a.I_off = obs->I_off;
    a.J_off = model->J_off;
    a.obs_p = (const float4*)obs->p;
    a.mod_c = (const float4*)model->center;
    a.mod_r = (const float4*)model->ray;
    a.mod_s = (const float4*)model->spot;
    a.obsX = (float4*)(ws + L.obsX);
    a.obsY = (float4*)(ws + L.obsY);
    a.modX = (float4*)(ws + L.modX);
    a.modY = (float4*)(ws + L.modY);
    a.modZ = (float4*)(ws + L.modZ);
    a.modW = (float4*)(ws + L.modW);
    a.I2_off = (int*)(ws + L.pairoff);
    a.J2_off = a.I2_off + (obs->T + 1);
    a.obs_gbase = a.J2_off + (obs->T + 1);
    a.mod_gbase = a.obs_gbase + (obs->T + 1);
    {
        size_t nsp = (size_t)obs->n + model->n + 2;
        int* pp = (int*)(ws + L.perm);
        // 2 (n_obs + 1) + 2 (n_model + 1) = 2 nsp ints
        a.obs_perm = pp;
        a.obs_pos = pp + obs->n + 1;
        a.mod_perm = pp + 2 * ((size_t)obs->n + 1);
        a.mod_pos = a.mod_perm + model->n + 1;
        a.sort_key = (unsigned*)(ws + L.sortbuf);
        a.sort_idx = (int*)(a.sort_key + 2 * nsp);
        a.obs_cone = (float4*)(ws + L.cone);
        a.mod_cone = a.obs_cone + L.max_obs_gran;
        a.obs_ext = (float*)(a.mod_cone + L.max_mod_gran);
        a.mod_ext = a.obs_ext + L.max_obs_gran;
        a.skip = h->skip;
    }
    a.row_tiles = (int4*)(ws + L.row_tiles);
    a.col_tiles = (int4*)(ws + L.col_tiles);
    a.ang_tiles = (int4*)(ws + L.ang);
    a.row_part = (float2*)(ws + L.row_part);
    a.col_part = (float2*)(ws + L.col_part);
    a.dust = (float*)(ws + L.dust);
    a.ctrl = (int*)(ws + L.ctrl);
    a.max_row_tiles = L.max_row_tiles;
    a.max_col_tiles = L.max_col_tiles;
    a.tile_rows = sk_variant_threads(h->row_variant);  // row pairs per tile (one per thread)
    a.tile_cols = sk_variant_threads(h->col_variant);
    double eps = prm->eps;
    a.negKD2 = (float)(-(double)geom->D * geom->D * 1.4426950408889634 / eps);
    {
        GeomDev G = laue_geom_dev(*geom);
        double dmin = geom->D;
        a.n_det = G.n_det;
        for (int k = 0; k < 4; ++k) {
            double Dk = k < G.n_det ? (double)G.Dd[k] : (double)geom->D;
            a.negK_det[k] = (float)(-Dk * Dk * 1.4426950408889634 / eps);
            if (k < G.n_det && Dk < dmin) dmin = Dk;
        }
        a.skipK = (float)(dmin * dmin * 1.4426950408889634 / eps);
    }
    a.kc = (float)((double)prm->c_out * 1.4426950408889634 / eps);
    a.frac = prm->unmatched_frac;
    a.to_user = (float)(eps * 0.6931471805599453);
    a.mode = prm->dust_mode == 2 ? 2 : (prm->dust_mode ? 1 : 0);
    a.tau_row = a.mode == 2 ? (float)((double)prm->kappa / ((double)prm->kappa + eps)) : 1.0f;
    a.tau_col = a.mode == 2 ? (float)((double)prm->lambda / ((double)prm->lambda + eps)) : 1.0f;
    a.warm = prm->warm_start ? 1 : 0;
    *out = a;
    lc->row_variant = h->row_variant;
    lc->col_variant = h->col_variant;
    int rt = std::max(1, std::min(h->sm_count * h->row_occ[h->row_variant], L.max_row_tiles));
    int ct = std::max(1, std::min(h->sm_count * h->col_occ[h->col_variant], L.max_col_tiles));
    lc->row_grid = rt;
    lc->col_grid = ct;
    // harvest passes: CTAs as wide as the tiles, about 768 threads per SM
    lc->hrv_grid = std::max(1, std::min(h->sm_count * (768 / a.tile_rows), L.max_row_tiles));
    lc->hcol_grid = std::max(1, std::min(h->sm_count * (768 / a.tile_cols), L.max_col_tiles));
    return LAUE_OK;
}

extern "C" int laue_cost_sinkhorn(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                                  const LaueModelSpots* model, const LaueOTParams* prm, float* f, float* g,
                                  float* dust, int* assign, float* margin, float* marg_err, float* q,
                                  void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (!prm || !(prm->eps > 0.0f) || prm->n_iter < 0 || !(prm->c_out >= 0.0f) ||
        !(prm->unmatched_frac >= 0.0) || prm->unmatched_frac > 1.0 || prm->dust_mode < 0 || prm->dust_mode > 2 ||
        (prm->dust_mode == 2 && (!(prm->kappa > 0.0f) || !(prm->lambda > 0.0f))))
        return laue_fail(h, LAUE_ERR_INVALID_ARG,
                         "OT params: eps > 0, n_iter >= 0, c_out >= 0, 0 <= frac <= 1, dust_mode 0..2, kappa and "
                         "lambda > 0 for the unbalanced mode");
    if (obs->T != model->T) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed and model T differ");
    if ((obs->n > 0 && !f) || (model->n > 0 && !g))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "f and g outputs are required");
    if (prm->warm_start && !dust) return laue_fail(h, LAUE_ERR_INVALID_ARG, "warm start needs dust");
    LaueProblemDims d{obs->T, obs->n, model->n, 0, 0, 0, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    SkArgs a;
    SkLaunch lc;
    laue_fill_sk(h, geom, obs, model, prm, L, &a, &lc);
    a.f = f;
    a.g = g;
    a.dust_out = dust;
    a.assign = assign;
    a.margin = margin;
    a.marg_err = marg_err;
    a.q = q;
    bool rows = assign || margin || marg_err;
    bool cols = q || marg_err;
    return laue_cuda_check(h, sinkhorn_run(a, lc, prm->n_iter, rows, cols, (cudaStream_t)stream),
                           "sinkhorn launch");
}

// ------------------------------------------------------- sparse Sinkhorn

extern "C" int laue_sparse_workspace_size(int T, int n_obs, int n_model, int rho, size_t* bytes) {
    if (!bytes || T < 1 || n_obs < 0 || n_model < 0 || rho < 1 || rho > kSparseMaxRho) return LAUE_ERR_INVALID_ARG;
    *bytes = kCtrlBytes + sparse_workspace_bytes(T, n_obs, n_model, rho);
    return LAUE_OK;
}

extern "C" int laue_cost_sinkhorn_sparse(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                                         const LaueModelSpots* model, const LaueOTParams* prm, int rho, float* f,
                                         float* g, float* dust, int* assign, float* margin, float* marg_err,
                                         float* q, int* nbr, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (!prm || !(prm->eps > 0.0f) || prm->n_iter < 0 || !(prm->c_out >= 0.0f) ||
        !(prm->unmatched_frac >= 0.0) || prm->unmatched_frac > 1.0 || prm->dust_mode < 0 || prm->dust_mode > 1)
        return laue_fail(h, LAUE_ERR_INVALID_ARG,
                         "sparse OT params: eps > 0, n_iter >= 0, c_out >= 0, 0 <= frac <= 1, dust_mode 0 or 1");
    if (rho < 1 || rho > kSparseMaxRho)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "rho must be 1..%d", kSparseMaxRho);
    if (obs->T != model->T) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed and model T differ");
    if ((obs->n > 0 && !f) || (model->n > 0 && !g))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "f and g outputs are required");
    if (prm->warm_start && !dust) return laue_fail(h, LAUE_ERR_INVALID_ARG, "warm start needs dust");
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    size_t need = kCtrlBytes + sparse_workspace_bytes(obs->T, obs->n, model->n, rho);
    if (need > h->ws_bytes)
        return laue_fail(h, LAUE_ERR_WORKSPACE, "sparse E-step: workspace of %zu bytes needed", need);
    SpArgs a{};
    sparse_carve(a, (char*)h->ws + kCtrlBytes, obs->T, obs->n, model->n, rho);
    a.T = obs->T;
    a.n_obs = obs->n;
    a.n_model = model->n;
    a.rho = rho;
    a.I_off = obs->I_off;
    a.J_off = model->J_off;
    a.p = (const float4*)obs->p;
    a.c = (const float4*)model->center;
    a.r = (const float4*)model->ray;
    a.s = (const float4*)model->spot;
    {
        GeomDev G = laue_geom_dev(*geom);
        a.n_det = G.n_det;
        for (int k = 0; k < 4; ++k) {
            float dr = k < G.n_det ? G.Dd[k] / geom->D : 1.0f;
            a.kdet[k] = dr * dr;
        }
    }
    a.ctrl = (int*)h->ws;
    const double eps = prm->eps;
    a.negK = (float)(-(double)geom->D * geom->D * 1.4426950408889634 / eps);
    a.kc = (float)((double)prm->c_out * 1.4426950408889634 / eps);
    a.frac = prm->unmatched_frac;
    a.to_user = (float)(eps * 0.6931471805599453);
    a.mode = prm->dust_mode;
    a.warm = prm->warm_start ? 1 : 0;
    a.f = f;
    a.g = g;
    a.dust_out = dust;
    a.assign = assign;
    a.margin = margin;
    a.marg_err = marg_err;
    a.q = q;
    a.nbr_out = nbr;
    bool rows = assign || margin || marg_err;
    bool cols = q || marg_err;
    return laue_cuda_check(h, sparse_sinkhorn_run(a, prm->n_iter, rows, cols, (cudaStream_t)stream),
                           "sparse sinkhorn launch");
}

// ------------------------------------------------------------- autotuner

extern "C" int laue_read_counters(laue_handle* h, void* stream, long long* counts_host, int n) {
    if (!h || !counts_host || n < 0 || n > 5) return LAUE_ERR_INVALID_ARG;
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned v[6] = {0u, 0u, 0u, 0u, 0u, 0u};  // exact rows, exact columns, fit pairs, pass pairs (64 bits)
    unsigned w[2] = {0u, 0u};                  // M-step pairs (64 bits)
    int* ctrl = (int*)h->ws;
    int rc;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(v, ctrl + CTRL_EXACT_ROWS, sizeof(v), cudaMemcpyDeviceToHost, s),
                              "reading counts")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(w, ctrl + CTRL_MS_PAIRS, sizeof(w), cudaMemcpyDeviceToHost, s),
                              "reading counts")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaMemsetAsync(ctrl + CTRL_EXACT_ROWS, 0, sizeof(v), s), "clearing counts")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaMemsetAsync(ctrl + CTRL_MS_PAIRS, 0, sizeof(w), s), "clearing counts")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "synchronise"))) return rc;
    long long all[5] = {(long long)v[0], (long long)v[1],
                        (long long)((unsigned long long)v[2] | ((unsigned long long)v[3] << 32)),
                        (long long)((unsigned long long)v[4] | ((unsigned long long)v[5] << 32)),
                        (long long)((unsigned long long)w[0] | ((unsigned long long)w[1] << 32))};
    for (int k = 0; k < n; ++k) counts_host[k] = all[k];
    return LAUE_OK;
}

extern "C" int laue_set_pair_skipping(laue_handle* h, int enable) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    h->skip = enable ? 1 : 0;
    return LAUE_OK;
}

extern "C" int laue_set_launch_shape(laue_handle* h, int row_shape, int col_shape) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (row_shape < 0 || row_shape >= kSkVariants || col_shape < 0 || col_shape >= kSkVariants)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "launch shape must be 0..%d", kSkVariants - 1);
    h->row_variant = row_shape;
    h->col_variant = col_shape;
    return LAUE_OK;
}

extern "C" int laue_autotune(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                             const LaueModelSpots* model, const LaueOTParams* prm, int n_iter, int* choice_host,
                             float* ms_host, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (!prm || !(prm->eps > 0.0f) || obs->T != model->T || n_iter < 1)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "autotune: bad parameters");
    LaueProblemDims d{obs->T, obs->n, model->n, 0, 0, 0, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)h->ws;
    float* f_tmp = (float*)(ws + L.fwd_blocks);  // scratch potentials beyond the E-step regions
    size_t need = L.fwd_blocks + sizeof(float) * ((size_t)obs->n + model->n + 2 * obs->T + 8);
    if (need > h->ws_bytes) return laue_fail(h, LAUE_ERR_WORKSPACE, "autotune: workspace too small");
    float* g_tmp = f_tmp + obs->n + 1;
    float* d_tmp = g_tmp + model->n + 1;
    cudaEvent_t e0, e1;
    if ((rc = laue_cuda_check(h, cudaEventCreate(&e0), "event"))) return rc;
    if ((rc = laue_cuda_check(h, cudaEventCreate(&e1), "event"))) return rc;
    float best_row = 3e38f, best_col = 3e38f;
    int row_v = 0, col_v = 0;
    int save_r = h->row_variant, save_c = h->col_variant;
    for (int v = 0; v < kSkVariants && rc == LAUE_OK; ++v) {
        // each shape with its own tile size: rebuild the schedule, warm up, time the passes
        h->row_variant = v;
        h->col_variant = v;
        SkArgs a;
        SkLaunch lc;
        laue_fill_sk(h, geom, obs, model, prm, L, &a, &lc);
        a.f = f_tmp;
        a.g = g_tmp;
        a.dust_out = d_tmp;
        a.warm = 0;
        if ((rc = laue_cuda_check(h, sinkhorn_prepare(a, s), "autotune prepare"))) break;
        sinkhorn_iterate(a, lc, 1, s);
        float ms = 0.0f;
        cudaEventRecord(e0, s);
        for (int k = 0; k < n_iter; ++k) sinkhorn_row_pass(a, lc, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_host) ms_host[2 * v] = ms / n_iter;
        if (ms < best_row) { best_row = ms; row_v = v; }
        cudaEventRecord(e0, s);
        for (int k = 0; k < n_iter; ++k) sinkhorn_col_pass(a, lc, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_host) ms_host[2 * v + 1] = ms / n_iter;
        if (ms < best_col) { best_col = ms; col_v = v; }
        rc = laue_cuda_check(h, cudaGetLastError(), "autotune passes");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LAUE_OK) {
        h->row_variant = save_r;
        h->col_variant = save_c;
        return rc;
    }
    h->row_variant = row_v;
    h->col_variant = col_v;
    if (choice_host) {
        choice_host[0] = row_v;
        choice_host[1] = col_v;
    }
    return LAUE_OK;
}

// ------------------------------------------------------------- not yet built

static int mstep_entry(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
                       const LaueModelSpots* model, const float* f, const float* g, const LaueMParams* prm,
                       const float* omega, float* R, float* x, int N, float* step_norms, void* stream, bool adjoint) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (obs->T != model->T) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed and model T differ");
    if (!prm || !(prm->eps > 0.0f) || prm->n_newton < 0 || prm->n_mm < 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "M-step params: eps > 0, n_newton >= 0, n_mm >= 0");
    if (!lat || lat->M < 1 || !lat->w_d0 || !aligned16(lat->w_d0))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "lattice: M >= 1 and aligned w_d0");
    if (N < 0 || (N > 0 && (!R || !x)) || !omega || (obs->n > 0 && !f) || (model->n > 0 && !g))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "M-step: NULL array or N < 0");
    LaueProblemDims d{obs->T, obs->n, model->n, N, lat->M, 0, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    MsArgs m{};
    SkLaunch lc;
    LaueOTParams op{0.4, prm->eps, 0.0f, 0, 0, 1, 0};
    laue_fill_sk(h, geom, obs, model, &op, L, &m.sk, &lc);
    // the M-step pair kernel runs one thread per column pair of the column
    // pass's tiles (narrow tiles skip more), about 768 threads per SM
    lc.col_grid = std::max(1, std::min(h->sm_count * (768 / m.sk.tile_cols), L.max_col_tiles));
    m.sk.f = const_cast<float*>(f);
    m.sk.g = const_cast<float*>(g);
    m.sk.dust_out = nullptr;
    m.sk.warm = 1;
    char* ws = (char*)h->ws;
    m.sk.dust = (float*)(ws + L.dust);
    m.w_d0 = (const float4*)lat->w_d0;
    m.M = lat->M;
    m.omega = omega;
    m.T = obs->T;
    m.N = N;
    m.n_model = model->n;
    m.J_off = model->J_off;
    m.grain = model->grain;
    m.plane = model->plane;
    m.angle = model->angle;
    m.R = R;
    m.x = x;
    m.jsum = (float*)(ws + L.jsum);
    m.seg = (int*)(ws + L.gidx);
    m.gstate = (float*)(ws + L.gsum);
    m.step_norms = step_norms;
    m.tol_x = prm->tol_x;
    m.tol_R = prm->tol_R;
    m.hreg = prm->hreg;
    m.n_newton = prm->n_newton;
    m.n_mm = prm->n_mm;
    for (int k = 0; k < 3; ++k) m.e[k] = geom->beam[k];
    m.D2 = geom->D * geom->D;
    {
        GeomDev G = laue_geom_dev(*geom);
        for (int k = 0; k < 4; ++k) m.D2det[k] = k < G.n_det ? G.Dd[k] * G.Dd[k] : m.D2;
    }
    if (adjoint)
        return laue_cuda_check(h, mstep_adjoint_run(m, lc, prm->n_newton, (cudaStream_t)stream),
                               "mstep_adjoint launch");
    return laue_cuda_check(h, mstep_run(m, lc, (cudaStream_t)stream), "mstep launch");
}

extern "C" int laue_mstep(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
                          const LaueModelSpots* model, const float* f, const float* g, const LaueMParams* prm,
                          const float* omega, float* R, float* x, int N, float* step_norms, void* stream) {
    return mstep_entry(h, geom, lat, obs, model, f, g, prm, omega, R, x, N, step_norms, stream, false);
}

extern "C" int laue_mstep_adjoint(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                                  const LaueObsSpots* obs, const LaueModelSpots* model, const float* f,
                                  const float* g, const LaueMParams* prm, const float* omega, float* R, float* x,
                                  int N, float* step_norms, void* stream) {
    if (prm && !(prm->hreg >= 0.0f)) return laue_fail(h, LAUE_ERR_INVALID_ARG, "mstep_adjoint: hreg >= 0");
    return mstep_entry(h, geom, lat, obs, model, f, g, prm, omega, R, x, N, step_norms, stream, true);
}

extern "C" int laue_objective_grad(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                                   const LaueObsSpots* obs, const LaueModelSpots* model, const float* f,
                                   const float* g, float eps, const float* omega, const float* R, const float* x,
                                   int N, float* grad, float* value, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if ((rc = laue_check_model(h, model))) return rc;
    if (obs->T != model->T) return laue_fail(h, LAUE_ERR_INVALID_ARG, "observed and model T differ");
    if (!(eps > 0.0f)) return laue_fail(h, LAUE_ERR_INVALID_ARG, "eps must be > 0");
    if (!lat || lat->M < 1 || !lat->w_d0 || !aligned16(lat->w_d0))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "lattice: M >= 1 and aligned w_d0");
    if (N < 0 || (N > 0 && (!R || !x || !grad)) || !omega || (obs->n > 0 && !f) || (model->n > 0 && !g))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "objective_grad: NULL array or N < 0");
    LaueProblemDims d{obs->T, obs->n, model->n, N, lat->M, 0, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    MsArgs m{};
    SkLaunch lc;
    LaueOTParams op{0.4, eps, 0.0f, 0, 0, 1, 0};
    laue_fill_sk(h, geom, obs, model, &op, L, &m.sk, &lc);
    // the M-step pair kernel runs one thread per column pair of the column
    // pass's tiles (narrow tiles skip more), about 768 threads per SM
    lc.col_grid = std::max(1, std::min(h->sm_count * (768 / m.sk.tile_cols), L.max_col_tiles));
    m.sk.f = const_cast<float*>(f);
    m.sk.g = const_cast<float*>(g);
    m.sk.dust_out = nullptr;
    m.sk.warm = 1;
    char* ws = (char*)h->ws;
    m.w_d0 = (const float4*)lat->w_d0;
    m.M = lat->M;
    m.omega = omega;
    m.T = obs->T;
    m.N = N;
    m.n_model = model->n;
    m.J_off = model->J_off;
    m.grain = model->grain;
    m.plane = model->plane;
    m.angle = model->angle;
    m.R = const_cast<float*>(R);
    m.x = const_cast<float*>(x);
    m.jsum = (float*)(ws + L.jsum);
    m.seg = (int*)(ws + L.gidx);
    m.gstate = (float*)(ws + L.gsum);
    for (int k = 0; k < 3; ++k) m.e[k] = geom->beam[k];
    m.D2 = geom->D * geom->D;
    {
        GeomDev G = laue_geom_dev(*geom);
        for (int k = 0; k < 4; ++k) m.D2det[k] = k < G.n_det ? G.Dd[k] * G.Dd[k] : m.D2;
    }
    m.grad = grad;
    m.value = value;
    return laue_cuda_check(h, grad_run(m, lc, (cudaStream_t)stream), "objective_grad launch");
}

extern "C" int laue_axis_angle(laue_handle* h, const float* w, const float* R0, float* R, float* JlT, int N,
                               void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (N < 0 || (N > 0 && (!w || !R0 || !R))) return laue_fail(h, LAUE_ERR_INVALID_ARG, "axis_angle: bad arguments");
    return laue_cuda_check(h, axis_angle_run(w, R0, R, JlT, N, (cudaStream_t)stream), "axis_angle launch");
}

extern "C" int laue_axis_angle_vjp(laue_handle* h, const float* w, const float* grad, const float* gout, float* gw,
                                   float* gx, int N, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (N < 0 || (N > 0 && (!w || !grad || !gw)))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "axis_angle_vjp: bad arguments");
    return laue_cuda_check(h, axis_angle_vjp_run(w, grad, gout, gw, gx, N, (cudaStream_t)stream),
                           "axis_angle_vjp launch");
}

extern "C" double laue_c_out(double sigma_mm, double D) {
    if (!(sigma_mm > 0.0) || !(D > 0.0)) return -1.0;
    return outlier_cost(sigma_mm, D);
}

extern "C" double laue_anneal_eps(double eps_final, int n_em, int k, double factor) {
    if (!(eps_final > 0.0) || n_em < 0 || k < 0 || !(factor > 0.0)) return -1.0;
    return anneal_eps(eps_final, n_em, k, factor);
}

extern "C" int laue_single_fit(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                               const LaueObsSpots* obs, const float* omega, const float* startR,
                               const float* startX, int S, const LaueSingleParams* prm, float* R_out,
                               float* x_out, int* keep, float* unmatched, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if (obs->T > kSfMaxT) return laue_fail(h, LAUE_ERR_INVALID_ARG, "single fit supports at most %d angles", kSfMaxT);
    if (!lat || lat->M < 1 || lat->M > 65535 || !lat->w_d0 || !lat->nharm || !aligned16(lat->w_d0))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "lattice: 1 <= M <= 65535 and aligned w_d0");
    if (!prm || !(prm->eps_final > 0.0f) || prm->k_max < 0 || prm->mstep.n_newton < 0 || prm->mstep.n_mm < 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "single-fit params: eps_final > 0, k_max >= 0");
    if (S < 0 || (S > 0 && (!startR || !startX || !R_out || !x_out || !keep)) || !omega)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "single fit: NULL array or S < 0");
    LaueProblemDims d{obs->T, obs->n, 0, 0, lat->M, 1, 0};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    char* ws = (char*)h->ws;
    SfArgs a{};
    a.G = laue_geom_dev(*geom);
    a.w_d0 = (const float4*)lat->w_d0;
    a.nharm = lat->nharm;
    a.M = lat->M;
    a.omega = omega;
    a.T = obs->T;
    a.I_off = obs->I_off;
    a.p = (const float4*)obs->p;
    a.R0 = startR;
    a.x0 = startX;
    a.S = S;
    a.R_out = R_out;
    a.x_out = x_out;
    a.keep = keep;
    a.unmatched = unmatched;
    a.eps_final = prm->eps_final;
    a.c_out = prm->c_out;
    a.f_out = prm->f_out;
    a.tol_x = prm->mstep.tol_x;
    a.tol_R = prm->mstep.tol_R;
    a.hreg = prm->mstep.hreg;
    a.k_max = prm->k_max;
    a.n_newton = prm->mstep.n_newton;
    a.n_mm = prm->mstep.n_mm;
    a.anneal = prm->anneal > 0.0f ? prm->anneal : 100.0f;
    a.recut = prm->recut;
    a.scratch = (float*)(ws + L.sfs);
    a.cap = kSfCap;
    a.icap = kSfIcap;
    a.ncap = (int)sf_near_cap(obs->n);
    a.ctrl = (int*)(ws + L.ctrl);
    a.queue = a.ctrl + CTRL_SF_NEXT;
    int ctas = h->sm_count * kSfCtasPerSm;
    return laue_cuda_check(h, single_fit_run(a, ctas, (cudaStream_t)stream), "single fit launch");
}

static SfArgs fill_sf(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
                      const float* omega, const float* R, const float* x, int S, float c_out, const Layout& L) {
    char* ws = (char*)h->ws;
    SfArgs a{};
    a.G = laue_geom_dev(*geom);
    a.w_d0 = (const float4*)lat->w_d0;
    a.nharm = lat->nharm;
    a.M = lat->M;
    a.omega = omega;
    a.T = obs->T;
    a.I_off = obs->I_off;
    a.p = (const float4*)obs->p;
    a.R0 = R;
    a.x0 = x;
    a.S = S;
    a.c_out = c_out;
    a.scratch = (float*)(ws + L.sfs);
    a.cap = kSfCap;
    a.icap = kSfIcap;
    a.ncap = (int)sf_near_cap(obs->n);
    a.ctrl = (int*)(ws + L.ctrl);
    a.queue = a.ctrl + CTRL_SF_NEXT;
    return a;
}

extern "C" int laue_prototype_select(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                                     const LaueObsSpots* obs, const float* omega, const float* candR,
                                     const float* candX, int Nc, float eps_s, float c_out, int k_max, int* order,
                                     float* gains, int* k_star_host, long long* nnz_host, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    if (obs->T > kSfMaxT) return laue_fail(h, LAUE_ERR_INVALID_ARG, "at most %d angles", kSfMaxT);
    if (!lat || lat->M < 1 || lat->M > 65535 || !lat->w_d0 || !lat->nharm || !aligned16(lat->w_d0))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "lattice: 1 <= M <= 65535 and aligned w_d0");
    if (Nc < 0 || k_max < 0 || (Nc > 0 && (!candR || !candX)) || (k_max > 0 && (!order || !gains)) ||
        !k_star_host || !omega || !(eps_s > 0.0f))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "prototype_select: bad arguments");
    LaueProblemDims d{obs->T, obs->n, 0, 0, lat->M, 1, Nc > 0 ? Nc : 1};
    Layout L;
    if ((rc = laue_need_ws(h, d, &L))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)h->ws;
    SfArgs a = fill_sf(h, geom, lat, obs, omega, candR, candX, Nc, c_out, L);
    SpotArgs sp{};
    int* ip = (int*)(ws + L.spot);
    sp.eps_s = eps_s;
    sp.count = ip;
    sp.row_ptr = ip + Nc;
    sp.chosen = sp.row_ptr + Nc + 1;
    int blocks = h->sm_count * 4;
    sp.part_i = sp.chosen + Nc;
    sp.part_g = (float*)(sp.part_i + blocks);
    sp.tick = (int*)(sp.part_g + blocks);
    sp.cur = sp.tick + 1;
    sp.kstar = sp.tick + 2;
    sp.nnz_total = (long long*)(((uintptr_t)(sp.tick + 4) + 7) & ~(uintptr_t)7);
    sp.best = (float*)(sp.nnz_total + 2);
    int ctas = h->sm_count * kSfCtasPerSm;
    if ((rc = laue_cuda_check(h, spot_matrix_run(a, sp, ctas, true, s), "spot count"))) return rc;
    long long nnz = 0;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(&nnz, sp.nnz_total, sizeof(long long), cudaMemcpyDeviceToHost, s),
                              "reading nnz")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "spot synchronise"))) return rc;
    if (nnz_host) *nnz_host = nnz;
    size_t tail = h->ws_bytes - L.total;
    if ((size_t)nnz * 8 + 512 > tail)
        return laue_fail(h, LAUE_ERR_CAPACITY, "prototype_select: %lld nonzeros need %zu more workspace bytes", nnz,
                         (size_t)nnz * 8 + 512 - tail);
    sp.col = (int*)(ws + L.total);
    sp.val = (float*)(ws + align_up(L.total + sizeof(int) * (size_t)nnz, 256));
    sp.order = order;
    sp.gains = gains;
    if ((rc = laue_cuda_check(h, spot_matrix_run(a, sp, ctas, false, s), "spot fill"))) return rc;
    if ((rc = laue_cuda_check(h, spot_greedy_run(sp, obs->n, Nc, k_max, h->sm_count, s), "spot greedy"))) return rc;
    int ks = 0;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(&ks, sp.kstar, sizeof(int), cudaMemcpyDeviceToHost, s),
                              "reading k*")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "spot synchronise"))) return rc;
    *k_star_host = ks;
    return LAUE_OK;
}
