// hostapi.h -- host helpers shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/swcorr.h"
#include "launch.h"

namespace swc {

struct DeviceInfo {
  int dev = -1;
  int sms = 0;
  int smem_optin = 0;
  int cc_major = 0, cc_minor = 0;
  char name[256] = {0};
};

// Record a detail message (swcorr_last_error) and return st.
swcorr_status fail(swcorr_status st, const char* fmt, ...);
swcorr_status cuda_fail(cudaError_t e, const char* what);

// Current device's attributes; SWCORR_ERR_NO_DEVICE unless it is sm_103.
swcorr_status device_info(DeviceInfo* d);

// 2-D tiled tensor map with boxes of box_w x 1 elements, zero fill outside.
swcorr_status encode_2d(CUtensorMap* m, CUtensorMapDataType dt, int elem_bytes, const void* base, int64_t W,
                        int64_t H, int64_t pitch_elems, int box_w);

// Geometry, launch shape and per-launch constants of the 2-D kernels.
// *tune holds the requested launch parameters (0 = default) on entry and the
// ones in use on return.
swcorr_status setup_2d(const DeviceInfo& dev, swcorr_dtype dt, int H, int W, int kh, int kw, int sy, int sx,
                       Geo2DInfo* g2, K2DParams* k2, size_t* smem_out, int* grid_out, swcorr_tune* tune);
swcorr_status bind_2d(K2DParams* k2, const Geo2DInfo& g2, swcorr_dtype dt, const void* x, const void* y, int64_t ip,
                      float* c, int64_t op, int64_t* sums, bool encode_maps, bool* use_tma);

// The same for the 2-D uint16 kernel (used by the no-allocation entry point).
swcorr_status setup_2d_u16(const DeviceInfo& dev, int H, int W, int kh, int kw, int sy, int sx, Geo2DInfo* g2,
                           K2DParams* k2, size_t* smem_out, int* grid_out);

// Bind buffers to a set-up 2-D uint16 launch (tensor maps encoded when
// encode_maps and the layout allows TMA); reports whether TMA is used.
swcorr_status bind_2d_u16(K2DParams* k2, const Geo2DInfo& g2, const void* x, const void* y, int64_t ip, float* c,
                          int64_t op, int64_t* sums, bool encode_maps, bool* use_tma);

// Tune cache (tune.cu): the entry for (device, kind "plain"/"batched", ndim,
// k, dtype) if the loaded cache has one; range check of explicit parameters.
bool tune_lookup(const char* device, const char* kind, int ndim, const int32_t* k, swcorr_dtype dtype,
                 swcorr_tune* out);
swcorr_status tune_check(const swcorr_tune* t);

}  // namespace swc
