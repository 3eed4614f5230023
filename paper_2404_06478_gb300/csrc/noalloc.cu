// noalloc.cu — laue_cost_sinkhorn_noalloc: the fused cost + Sinkhorn E-step
// for callers that cannot allocate device memory.
//
// Its scratch is a fixed array in device memory that belongs to this library
// module: it is reserved when the module loads on a GPU and held there until
// the process exits.  Host code never dereferences or launches with the
// array's name (on the host that name is only a stand-in for the device
// symbol); the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and that address is what
// the kernels receive.
#include <mutex>

#include "api_internal.h"

namespace laue {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

}  // namespace laue

using namespace laue;

namespace {

constexpr int kMaxDevices = 64;

struct StaticDevice {
    bool ready;
    int device;     // CUDA ordinal this entry describes
    void* scratch;  // device address of g_static_scratch on this device
    int sm_count;
    int row_occ[kSkVariants], col_occ[kSkVariants];
};

StaticDevice g_devices[kMaxDevices];
std::mutex g_setup_mutex;

// One-time set-up for the current device: the device address of the static
// scratch, the SM count and the occupancy of the pair passes.
int static_device(StaticDevice** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LAUE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    StaticDevice& d = g_devices[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return LAUE_ERR_CUDA;
        int sm = 0;
        if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LAUE_ERR_CUDA;
        if (sinkhorn_occupancy(d.row_occ, d.col_occ) != 0)
            for (int v = 0; v < kSkVariants; ++v) d.row_occ[v] = d.col_occ[v] = 1;
        d.device = dev;
        d.scratch = p;
        d.sm_count = sm;
        d.ready = true;
    }
    *out = &d;
    return LAUE_OK;
}

}  // namespace

extern "C" int laue_cost_sinkhorn_noalloc(const LaueGeometry* geom, const LaueObsSpots* obs,
                                          const LaueModelSpots* model, const LaueOTParams* prm, float* f, float* g,
                                          float* dust, int* assign, float* margin, float* marg_err, float* q,
                                          int* status, void* stream) {
    int rc;
    if ((rc = laue_check_geom(nullptr, geom))) return rc;
    if ((rc = laue_check_obs(nullptr, obs))) return rc;
    if ((rc = laue_check_model(nullptr, model))) return rc;
    if (!prm || !(prm->eps > 0.0f) || prm->n_iter < 0 || !(prm->c_out >= 0.0f) || !(prm->unmatched_frac >= 0.0) ||
        prm->unmatched_frac > 1.0 || obs->T != model->T || (obs->n > 0 && !f) || (model->n > 0 && !g) ||
        prm->dust_mode < 0 || prm->dust_mode > 2 ||
        (prm->dust_mode == 2 && (!(prm->kappa > 0.0f) || !(prm->lambda > 0.0f))) ||
        (prm->warm_start && !dust))
        return LAUE_ERR_INVALID_ARG;
    StaticDevice* d = nullptr;
    if ((rc = static_device(&d))) return rc;
    // the E-step uses the layout regions in front of the forward-model scratch
    LaueProblemDims dims{obs->T, obs->n, model->n, 0, 0, 0, 0};
    Layout L = make_layout(dims, d->sm_count);
    if (L.fwd_blocks > kStaticScratchBytes) return LAUE_ERR_CAPACITY;
    laue_handle h{};  // a view of the static scratch; nothing is allocated
    h.device = d->device;
    h.sm_count = d->sm_count;
    for (int v = 0; v < kSkVariants; ++v) {
        h.row_occ[v] = d->row_occ[v];
        h.col_occ[v] = d->col_occ[v];
    }
    h.row_variant = h.col_variant = kSkDefaultVariant;
    h.skip = 1;
    h.ws = d->scratch;
    h.ws_bytes = kStaticScratchBytes;
    cudaStream_t s = (cudaStream_t)stream;
    // counters and the status word must start at zero: the array keeps the
    // previous call's contents
    if (cudaMemsetAsync(d->scratch, 0, kCtrlBytes, s) != cudaSuccess) return LAUE_ERR_CUDA;
    SkArgs a;
    SkLaunch lc;
    laue_fill_sk(&h, geom, obs, model, prm, L, &a, &lc);
    a.f = f;
    a.g = g;
    a.dust_out = dust;
    a.assign = assign;
    a.margin = margin;
    a.marg_err = marg_err;
    a.q = q;
    bool rows = assign || margin || marg_err;
    bool cols = q || marg_err;
    if (sinkhorn_run(a, lc, prm->n_iter, rows, cols, s) != cudaSuccess) return LAUE_ERR_CUDA;
    if (status && cudaMemcpyAsync(status, (char*)d->scratch + sizeof(int) * CTRL_STATUS, sizeof(int),
                                  cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LAUE_ERR_CUDA;
    return LAUE_OK;
}
