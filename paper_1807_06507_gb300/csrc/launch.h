// launch.h -- host-side entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "kparams.h"
#include "k1d_params.h"

namespace swc {

struct Geo2DInfo {
  int M, KW, HALO, RW, RWS, TAIL;
};

// 2-D uint16: geometry of the instance that serves window width kw (false if
// kw has no instance) and its launch.
bool k2d_u16_geometry(int kw, Geo2DInfo* g);
cudaError_t k2d_u16_launch(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma);
// resident CTAs per SM of that instance (32-bit or 64-bit second moments)
// with `smem` bytes of dynamic shared memory; 0 if the query fails
int k2d_u16_blocks_per_sm(int kw, bool wide, size_t smem);

// 2-D float32: same interface.
bool k2d_f32_geometry(int kw, Geo2DInfo* g);
// tier: the float32 second tier's placement (0 in place, 1 listed as tasks,
// 2 the listed tasks; k2d_f32.cuh)
cudaError_t k2d_f32_launch(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier = 0);
// the instances of eight pairs of window widths (1-3, 5-7, ..., 29-31)
cudaError_t k2d_f32_launch_p0(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p1(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p2(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p3(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p4(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p5(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p6(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);
cudaError_t k2d_f32_launch_p7(int kw, const K2DParams& p, int grid, size_t smem, cudaStream_t st, bool tma, int tier);

// 1-D (uint16 or float32): outputs per lane per chunk, and the launch.
int k1d_outputs_per_lane();
cudaError_t k1d_launch(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st);
// float32 second tier: the wide form over the chunks the first launch listed
cudaError_t k1d_wide_launch(const K1DParams& p, int grid, int warps, size_t smem, cudaStream_t st);
// resident CTAs of `warps` warps per SM with `smem` bytes (0 if the query fails)
int k1d_blocks_per_sm(bool f32, int warps, size_t smem);

// Batched 2-D uint16: ring row stride, one-time attribute set-up, launch.
int kbatched_ring_row();
// Batched kernel classes: 0 = 32-bit engine, 1 = 64-bit up to 17 columns, 2 = 64-bit above.
const void* kbatched_kernel_ptr(int cls);
cudaError_t kbatched_prepare();
cudaError_t kbatched_launch(const KBatchParams& p, int cls, int grid, size_t smem, cudaStream_t st);

// Batched 2-D float32: ring row stride, kernel (occupancy queries), launch.
int kbatched_f32_ring_row();
const void* kbatched_f32_kernel_ptr(int cls);
cudaError_t kbatched_f32_prepare();
// the instances of two groups of window widths (1-15, 17-31), by width
const void* kbatched_f32_kernel_ptr_p0(int kw);
const void* kbatched_f32_kernel_ptr_p1(int kw);
cudaError_t kbatched_f32_launch_p0(int kw, const KBatchParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t kbatched_f32_launch_p1(int kw, const KBatchParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t kbatched_f32_launch(const KBatchParams& p, int cls, int grid, size_t smem, cudaStream_t st);

// 3-D (uint16 or float32), square in-plane windows ky = kx = k.
struct Geo3DInfo {
  int TY, TX, TYI, BXW, XH, VSP;
};
struct K3DParams;
bool k3d_geometry(int k, Geo3DInfo* g);
cudaError_t k3d_launch(int k, const K3DParams& p, int grid, size_t smem, cudaStream_t st);
// float32 second tier: the wide kernel over the items the first launch listed
cudaError_t k3d_wide_launch(int k, const K3DParams& p, int grid, size_t smem, cudaStream_t st);
// resident CTAs per SM of that instance with `smem` bytes (0 if the query fails)
int k3d_blocks_per_sm(int k, size_t smem);

}  // namespace swc
