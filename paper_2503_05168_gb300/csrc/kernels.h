// kernels.h -- host-side launchers of the Seele kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace seele {

void launch_repack(int n, int nc, const float* means, const float* log_scales, const float* quats,
                   const float* logits, const float* sh, float4* pos_logit, float4* quat, float4* log_scale,
                   float4* shp, cudaStream_t s);

void launch_preprocess(const SceneDev& sc, const CamDev* cams, const FrameParams& fp, const ProjOut& out,
                       cudaStream_t s);

uint32_t scan_tiles_per_launch();
void launch_compact_visible(const uint32_t* tiles, const float* depth, uint32_t R, uint32_t* keys, uint32_t* vals,
                            uint64_t* status, uint32_t epoch, DeviceStatus* st, int ticket, cudaStream_t s);
void launch_scan_tiles(const uint32_t* tiles, const uint32_t* order, uint32_t max_n, uint32_t* offsets,
                       uint64_t* status, uint32_t epoch, DeviceStatus* st, int ticket, uint32_t capacity,
                       cudaStream_t s);

uint32_t sort_tile_items();
void launch_radix_histogram(const uint32_t* keys, const uint32_t* count_ptr, int passes, uint32_t* hist,
                            int blocks, cudaStream_t s);
void launch_onesweep(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                     const uint32_t* count_ptr, uint32_t max_n, int shift, const uint32_t* hist, uint64_t* status,
                     uint32_t epoch, DeviceStatus* st, int ticket, cudaStream_t s);

void launch_emit(const uint32_t* order, const uint32_t* offsets, const uint2* rect, const CamDev* cams, int n_gauss,
                 const DeviceStatus* st, uint32_t* inst_tile, uint32_t* inst_rec, int blocks, cudaStream_t s);
void launch_ranges(const uint32_t* inst_tile, const DeviceStatus* st, uint2* ranges, int blocks, cudaStream_t s);

struct RasterArgs {
    const uint2* ranges;
    const uint32_t* inst_rec;
    const float4* rec;
    const CamDev* cams;
    int n_cams;
    uint32_t n_tiles;
    FrameParams fp;
    bool cr;
    int group_w, group_h;
    float* out_rgb;
    float* out_T;
    uint32_t* out_nc;
    DeviceStatus* count_into;   // non-null: run the counting variant
};
bool launch_raster_fwd(const RasterArgs& a, cudaStream_t s);

}  // namespace seele
