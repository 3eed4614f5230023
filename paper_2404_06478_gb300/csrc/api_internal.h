// api_internal.h — handle and host helpers shared by the C-ABI sources.
#pragma once

#include <cuda_runtime.h>

#include "../../include/laueot.h"
#include "common.cuh"
#include "kernels.h"

struct laue_handle {
    int device;
    int sm_count;
    int row_occ[laue::kSkVariants], col_occ[laue::kSkVariants];  // resident CTAs per SM of each launch shape
    int row_variant, col_variant;  // launch shapes in use (the autotuner's choice)
    int skip;                      // exact underflow skipping in the pair passes (default on)
    void* ws;
    size_t ws_bytes;
    char err[512];
};

int laue_fail(laue_handle* h, int code, const char* fmt, ...);
int laue_cuda_check(laue_handle* h, cudaError_t e, const char* what);
laue::GeomDev laue_geom_dev(const LaueGeometry& g);
int laue_check_geom(laue_handle* h, const LaueGeometry* g);
int laue_check_obs(laue_handle* h, const LaueObsSpots* o);
int laue_check_model(laue_handle* h, const LaueModelSpots* m);
int laue_need_ws(laue_handle* h, const LaueProblemDims& d, laue::Layout* L);
int laue_fill_sk(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs, const LaueModelSpots* model,
                 const LaueOTParams* prm, const laue::Layout& L, laue::SkArgs* out, laue::SkLaunch* lc);
