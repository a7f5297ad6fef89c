// plan.cu -- host side of libswcorr: argument validation, plans, TMA tensor
// maps, launches and the C ABI declared in include/swcorr.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/swcorr.h"
#include "hostapi.h"
#include "k3d.cuh"
#include "knd.h"
#include "launch.h"

using namespace swc;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace swc {

swcorr_status fail(swcorr_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

swcorr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SWCORR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace swc

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda
// link dependency).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

namespace swc {

swcorr_status encode_2d(CUtensorMap* m, CUtensorMapDataType dt, int elem_bytes, const void* base, int64_t W,
                        int64_t H, int64_t pitch_elems, int box_w) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch_elems * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)box_w, 1u};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return SWCORR_OK;
}

swcorr_status encode_1d(CUtensorMap* m, CUtensorMapDataType dt, const void* base, int64_t N) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[1] = {(cuuint64_t)N};
  cuuint64_t strides[1] = {0};
  cuuint32_t box[1] = {256u};
  cuuint32_t estr[1] = {1u};
  CUresult r = fn(m, dt, 1, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled (1-D) failed (CUresult %d)", (int)r);
  return SWCORR_OK;
}

swcorr_status encode_3d(CUtensorMap* m, CUtensorMapDataType dt, int eb, const void* base, int64_t W, int64_t H,
                        int64_t Z, int64_t py, int64_t pz, int box_w, int box_h) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)Z};
  cuuint64_t strides[2] = {(cuuint64_t)(py * eb), (cuuint64_t)(pz * eb)};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SWCORR_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (CUresult %d)", (int)r);
  return SWCORR_OK;
}

// Device name (cached per device ordinal).
static void device_name(int dev, char* out, size_t n) {
  static std::mutex mu;
  static std::map<int, std::string> names;
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it == names.end()) {
    cudaDeviceProp prop;
    std::string nm = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? std::string(prop.name) : std::string();
    it = names.emplace(dev, nm).first;
  }
  std::snprintf(out, n, "%s", it->second.c_str());
}

swcorr_status device_info(DeviceInfo* d) {
  cudaError_t e = cudaGetDevice(&d->dev);
  if (e != cudaSuccess) return fail(SWCORR_ERR_NO_DEVICE, "no CUDA device: %s", cudaGetErrorString(e));
  cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, d->dev);
  cudaDeviceGetAttribute(&d->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->dev);
  cudaDeviceGetAttribute(&d->cc_major, cudaDevAttrComputeCapabilityMajor, d->dev);
  cudaDeviceGetAttribute(&d->cc_minor, cudaDevAttrComputeCapabilityMinor, d->dev);
  device_name(d->dev, d->name, sizeof(d->name));
  if (d->cc_major != 10 || d->cc_minor != 3)
    return fail(SWCORR_ERR_NO_DEVICE, "libswcorr is built for sm_103a; device %d is sm_%d%d", d->dev, d->cc_major,
                d->cc_minor);
  return SWCORR_OK;
}

// Largest in-bounds window (cells) of the uint16 paths: the sum of a window's
// values stays below 2^31 (n * 65535 < 2^31) and n^2 * var below 2^62.
static constexpr uint64_t kMaxU16Cells = 32768;

// Fixed-point magnitude bits of the float32 paths for windows of n cells:
// |X| <= 2^qbits per cell, so n * 2^qbits < 2^31 keeps the window sums in
// int32 and n^2 (2^qbits)^2 < 2^62 keeps the int64 finalize exact; at most
// 22 bits (the rounding constant 1.5 * 2^23 of the conversion).
static int f32_qbits(uint64_t n) {
  int qb = 22;
  while (qb > 1 && (double)n * std::ldexp(1.0, qb) >= 2147483648.0) qb--;
  return qb;
}

// Fixed-point bits of the 3-D float32 kernel, whose first-moment sums are
// 64-bit: |X| < 2^q / 1.015625 + 1 (the map's margin and rounding), so
// n (2^q / 1.015625 + 1) < 2^31.5 keeps n^2 var(X), the bound of
// n Sxx - Sx^2 and of |n Sxy - Sx Sy|, below 2^63; the window sums of one
// plane (ky kx cells) stay below 2^31; at most 22 bits.
static int f32_qbits_3d(uint64_t n, uint64_t plane) {
  int qb = 22;
  auto mx = [&](int q) { return std::ldexp(1.0, q) / 1.015625 + 1.0; };
  while (qb > 1 && ((double)n * mx(qb) >= 3.03e9 || (double)plane * mx(qb) >= 2147483648.0)) qb--;
  return qb;
}

// Geometry, launch shape and per-launch constants of the 2-D kernels.
swcorr_status setup_2d(const DeviceInfo& dev, swcorr_dtype dt, int H, int W, int kh, int kw, int sy, int sx,
                       Geo2DInfo* g2, K2DParams* k2, size_t* smem_out, int* grid_out, swcorr_tune* tune) {
  const bool f32 = dt == SWCORR_F32;
  if (!(f32 ? k2d_f32_geometry(kw, g2) : k2d_u16_geometry(kw, g2)))
    return fail(SWCORR_ERR_UNSUPPORTED, "2-D %s: window width %d has no kernel instance (1..31 odd)",
                f32 ? "float32" : "uint16", kw);
  const Geo2DInfo& g = *g2;
  if (!f32 && (uint64_t)std::min(kh, H) * (uint64_t)std::min(kw, W) > kMaxU16Cells)
    return fail(SWCORR_ERR_UNSUPPORTED, "uint16 windows are limited to %llu in-bounds cells (got %d x %d)",
                (unsigned long long)kMaxU16Cells, kh, kw);
  Scene2D& sc = k2->sc;
  sc.H = H;
  sc.W = W;
  sc.kh = kh;
  sc.h1 = (kh - 1) / 2;
  sc.h2 = kh / 2;
  sc.kw = kw;
  sc.sy = sy;
  sc.sx = sx;
  sc.OH = (H + sy - 1) / sy;
  sc.OW = (W + sx - 1) / sx;
  sc.n_strips = (W + 32 * g.M - 1) / (32 * g.M);
  const uint64_t n = (uint64_t)kh * (uint64_t)kw;
  sc.inv_n = n <= 1 ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / n);
  sc.qbits = f32_qbits(n);
  // uint16 windows with more than 64 cells routinely have second moments
  // beyond 2^32: use the 64-bit engine there
  sc.wide = (!f32 && n > 64) ? 1 : 0;
  // rings of entering and leaving rows (x and y), PF + 1 slots each
  const int PF = tune->prefetch > 0 ? tune->prefetch : (f32 ? 3 : 4);
  const int NR = PF + 1;
  k2->NR = NR;
  k2->PF = PF;
  const size_t smem = (size_t)NR * g.RWS * (f32 ? 4 : 2) * 4 + (size_t)NR * 8;
  if (smem > (size_t)dev.smem_optin)
    return fail(SWCORR_ERR_UNSUPPORTED, "window height %d needs %zu B of shared memory", kh, smem);
  int per_sm = std::max(1, std::min(16, (int)((200 * 1024) / (smem + 1024))));
  if (!f32) {
    const int b = k2d_u16_blocks_per_sm(kw, sc.wide != 0, smem);
    if (b > 0) per_sm = std::min(per_sm, b);
  }
  if (tune->ctas_per_sm > 0) per_sm = std::min(per_sm, tune->ctas_per_sm);
  const int total = dev.sms * per_sm;
  // one wave of work items over the resident warps, but tiles at least
  // tile_rows tall (default 2 kh rows: the halo re-read stays below half)
  const int rows_min = tune->tile_rows > 0 ? tune->tile_rows : std::max(16, 2 * kh / std::max(1, sc.sy));
  int TJ = (int)((sc.OH * (int64_t)sc.n_strips + total - 1) / total);
  TJ = std::max(TJ, rows_min);
  TJ = std::min(TJ, sc.OH);
  sc.TJ = TJ;
  tune->prefetch = PF;
  tune->tile_rows = rows_min;
  tune->ctas_per_sm = per_sm;
  sc.n_rb = (sc.OH + TJ - 1) / TJ;
  k2->n_items = sc.n_rb * sc.n_strips;
  *grid_out = std::min(k2->n_items, total);
  *smem_out = smem;
  return SWCORR_OK;
}

swcorr_status setup_2d_u16(const DeviceInfo& dev, int H, int W, int kh, int kw, int sy, int sx, Geo2DInfo* g2,
                           K2DParams* k2, size_t* smem_out, int* grid_out) {
  swcorr_tune defaults{};
  return setup_2d(dev, SWCORR_U16, H, W, kh, kw, sy, sx, g2, k2, smem_out, grid_out, &defaults);
}

// Pointers, pitches and (when the layout allows TMA) tensor maps of one 2-D
// uint16 run; sets *use_tma.
swcorr_status bind_2d(K2DParams* k2, const Geo2DInfo& g2, swcorr_dtype dt, const void* x, const void* y, int64_t ip,
                      float* c, int64_t op, int64_t* sums, bool encode_maps, bool* use_tma) {
  const Scene2D& sc0 = k2->sc;
  const int64_t W = sc0.W, H = sc0.H;
  const int eb = dt == SWCORR_F32 ? 4 : 2;
  const CUtensorMapDataType tdt = dt == SWCORR_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  const bool base_ok = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  // TMA needs 16-byte aligned bases and row pitches; anything else takes the
  // plain-load row loader (same kernel, same results).
  *use_tma = base_ok && (ip * eb) % 16 == 0;
  if (*use_tma && encode_maps) {
    swcorr_status s1 = encode_2d(&k2->tmx, tdt, eb, x, W, H, ip, 256);
    if (s1 == SWCORR_OK) s1 = encode_2d(&k2->tmy, tdt, eb, y, W, H, ip, 256);
    if (s1 == SWCORR_OK && g2.TAIL > 0) {
      s1 = encode_2d(&k2->tmx_t, tdt, eb, x, W, H, ip, g2.TAIL);
      if (s1 == SWCORR_OK) s1 = encode_2d(&k2->tmy_t, tdt, eb, y, W, H, ip, g2.TAIL);
    }
    if (s1 != SWCORR_OK) return s1;
  }
  Scene2D& sc = k2->sc;
  sc.gx = x;
  sc.gy = y;
  sc.in_pitch = ip;
  sc.out = c;
  sc.out_pitch = op;
  sc.sums = reinterpret_cast<long long*>(sums);
  sc.vec_store = (sc.sx == 1 && (reinterpret_cast<uintptr_t>(c) & 15) == 0 && (op % 4) == 0) ? 1 : 0;
  return SWCORR_OK;
}

swcorr_status bind_2d_u16(K2DParams* k2, const Geo2DInfo& g2, const void* x, const void* y, int64_t ip, float* c,
                          int64_t op, int64_t* sums, bool encode_maps, bool* use_tma) {
  return bind_2d(k2, g2, SWCORR_U16, x, y, ip, c, op, sums, encode_maps, use_tma);
}

}  // namespace swc

constexpr int kMaxBatchClasses = 16;

enum PlanKind { KIND_2D_U16 = 1, KIND_2D_F32 = 2, KIND_1D = 3, KIND_3D = 4, KIND_ND = 5, KIND_BATCHED = 10 };

struct swcorr_plan_s {
  int kind = 0;
  int ndim = 0;
  int64_t shape[KND_MAXDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  int32_t k[KND_MAXDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  int32_t stride[KND_MAXDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  int64_t oshape[KND_MAXDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  swcorr_border border = SWCORR_BORDER_CLIP;
  swcorr_dtype dtype = SWCORR_U16;
  uint32_t flags = 0;
  DeviceInfo dev;
  swcorr_tune tune{};  // launch parameters in use (after defaults and the tune cache)
  // 2-D geometry and launch shape
  Geo2DInfo g2{};
  K2DParams k2{};
  int grid = 0;
  size_t smem = 0;
  // 1-D launch
  K1DParams k1{};
  int warps = 1;  // warps per CTA
  // 3-D launch
  K3DParams k3{};
  Geo3DInfo g3{};
  // general n-D path: parameters and its device block (two stream buffers,
  // scratch)
  KNDParams kn{};
  void* d_nd = nullptr;
  // the paper's -2 convention on a fused kernel: the fused run, then the
  // general path's mask-only pass (its missing-count buffers in d_mask)
  bool paper_post = false;
  KNDParams kmask{};
  void* d_mask = nullptr;
  // tensor-map cache
  const void* cached_x = nullptr;
  const void* cached_y = nullptr;
  int64_t cached_pitch = -1;
  // device status block
  uint32_t* d_status = nullptr;
  // float32 3-D plans: count and list of the items left to the wide kernel;
  // float32 2-D plans: count and list of the second-tier tasks
  int* d_redo = nullptr;
  // batched plans: device block (scenes, tensor maps, items, counter), graph
  void* d_batch = nullptr;
  // launches per kernel class: uint16 3 (32-bit engine; 64-bit up to 17
  // columns; 64-bit wider), float32 16 (one per window width)
  KBatchParams kbs[kMaxBatchClasses]{};
  int bgrid[kMaxBatchClasses] = {};
  int n_cls = 0;
  int64_t batched_outputs = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  // staging for host runs
  void* d_x = nullptr;
  void* d_y = nullptr;
  float* d_c = nullptr;
  // banded host runs of 2-D plans: input copies, band kernels, output copies
  // (kBands bands on the stream path, kGraphBands in the recorded graph)
  static constexpr int kBands = 8;
  static constexpr int kGraphBands = 5;
  static constexpr int kMaxBands = 16;
  cudaStream_t hs_in = nullptr, hs_out = nullptr, hs_cap = nullptr;
  cudaStream_t hs_k[kBands] = {};
  cudaEvent_t he_start = nullptr, he_done = nullptr;
  cudaEvent_t he_in[kMaxBands] = {}, he_k[kMaxBands] = {};
  // the recorded host-run graph and the host buffers it was recorded for
  cudaGraphExec_t hgraph_exec = nullptr;
  const void* hg_x = nullptr;
  const void* hg_y = nullptr;
  const void* hg_c = nullptr;
  bool hg_tma = false;
};

static int64_t n_outputs(const swcorr_plan_s* p) {
  if (p->kind == KIND_BATCHED) return p->batched_outputs;
  int64_t n = 1;
  for (int d = 0; d < p->ndim; d++) n *= p->oshape[d];
  return n;
}

static size_t elem_size(swcorr_dtype dt) { return dt == SWCORR_U16 ? 2 : 4; }

static swcorr_status plan_1d(swcorr_plan_s* p) {
  K1DParams& k1 = p->k1;
  const int64_t N = p->shape[0];
  const int k = p->k[0], s = p->stride[0];
  const int M1 = k1d_outputs_per_lane();
  const int L = 32 * M1;
  const int64_t seg = (int64_t)M1 * s;
  const int64_t q = k / seg;
  if (q > 31)
    return fail(SWCORR_ERR_UNSUPPORTED, "1-D window %d longer than 32 * %d * stride", k, M1);
  k1.N = N;
  k1.k = k;
  k1.h1 = (k - 1) / 2;
  k1.h2 = k / 2;
  k1.stride = s;
  k1.n_out = (N + s - 1) / s;
  k1.q = (int)q;
  k1.r = (int)(k % seg);
  k1.nseg = (int)std::min<int64_t>(64, 32 + q + 1);
  k1.is_f32 = p->dtype == SWCORR_F32 ? 1 : 0;
  if (!k1.is_f32 && (uint64_t)std::min<int64_t>(k, N) > kMaxU16Cells)
    return fail(SWCORR_ERR_UNSUPPORTED, "uint16 windows are limited to %llu in-bounds cells (got %d)",
                (unsigned long long)kMaxU16Cells, k);
  k1.qbits = f32_qbits((uint64_t)k);
  const int es = k1.is_f32 ? 4 : 2;
  const int align = 16 / es;
  // warps per CTA (one chunk of warps * 32 * M1 outputs shares one span):
  // the most (up to 4, or tile_rows when tuned) whose span fits in 110 KB
  auto smem_for = [&](int w, int* nbox) -> size_t {
    const int64_t need = align + (int64_t)(w - 1) * L * s + (int64_t)k1.nseg * seg;  // last warp's segments
    *nbox = (int)((need + 255) / 256);
    // (the span, at least w * L cells of two channels, also stages the w * L
    // float outputs)
    return (size_t)2 * (*nbox) * 256 * es + 8 + 16 * (size_t)w;
  };
  int warps = p->tune.tile_rows > 0 ? std::min(p->tune.tile_rows, 4) : 4;
  int nbox = 0;
  while (warps > 1 && smem_for(warps, &nbox) > (size_t)std::min(p->dev.smem_optin, 110 * 1024)) warps--;
  if ((size_t)2 * nbox * 256 * es < (size_t)warps * L * 4)
    return fail(SWCORR_ERR_UNSUPPORTED, "1-D span too short to stage the outputs");
  p->smem = smem_for(warps, &nbox);
  if (p->smem > (size_t)p->dev.smem_optin)
    return fail(SWCORR_ERR_UNSUPPORTED, "1-D window %d with stride %d needs %zu B of shared memory", k, s, p->smem);
  k1.nbox = nbox;
  k1.span = nbox * 256;
  k1.n_items = (k1.n_out + (int64_t)warps * L - 1) / ((int64_t)warps * L);
  p->warps = warps;
  int per_sm = k1d_blocks_per_sm(k1.is_f32 != 0, warps, p->smem);
  if (per_sm < 1) per_sm = 1;
  if (p->tune.ctas_per_sm > 0) per_sm = std::min(per_sm, p->tune.ctas_per_sm);
  p->grid = (int)std::min<int64_t>(k1.n_items, (int64_t)p->dev.sms * per_sm);
  p->tune.prefetch = 1;
  p->tune.tile_rows = warps;
  p->tune.ctas_per_sm = per_sm;
  return SWCORR_OK;
}

static swcorr_status run_1d(swcorr_plan_s* p, const void* x, const void* y, float* c, cudaStream_t st) {
  K1DParams& k1 = p->k1;
  const size_t es = elem_size(p->dtype);
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (es - 1))
    return fail(SWCORR_ERR_ALIGNMENT, "x and y must be aligned to their element size");
  const bool tma = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  if (tma) {
    if (x != p->cached_x || y != p->cached_y) {
      const CUtensorMapDataType dt =
          p->dtype == SWCORR_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
      swcorr_status s1 = encode_1d(&k1.tmx, dt, x, k1.N);
      if (s1 == SWCORR_OK) s1 = encode_1d(&k1.tmy, dt, y, k1.N);
      if (s1 != SWCORR_OK) {
        p->cached_x = p->cached_y = nullptr;
        return s1;
      }
      p->cached_x = x;
      p->cached_y = y;
    }
    k1.gx = k1.gy = nullptr;
  } else {
    k1.gx = x;
    k1.gy = y;
  }
  k1.rx = x;
  k1.ry = y;
  k1.out = c;
  k1.status = p->d_status;
  cudaError_t e;
  if (p->dtype == SWCORR_F32) {
    // chunks the chunk map leaves uncertified go to the wide launch
    k1.redo_count = p->d_redo;
    k1.redo_items = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(p->d_redo) + 8);
    if ((e = cudaMemsetAsync(p->d_redo, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "1-D chunk list reset");
  } else {
    k1.redo_count = nullptr;
    k1.redo_items = nullptr;
  }
  e = k1d_launch(k1, p->grid, p->warps, p->smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "1-D kernel launch");
  if (p->dtype == SWCORR_F32 && (e = k1d_wide_launch(k1, p->grid, p->warps, p->smem, st)) != cudaSuccess)
    return cuda_fail(e, "1-D wide kernel launch");
  return SWCORR_OK;
}

static swcorr_status plan_3d(swcorr_plan_s* p) {
  K3DParams& k3 = p->k3;
  if (p->k[1] != p->k[2])
    return fail(SWCORR_ERR_UNSUPPORTED, "3-D windows need equal row and column sizes (got %d x %d)", p->k[1],
                p->k[2]);
  if (!k3d_geometry(p->k[2], &p->g3))
    return fail(SWCORR_ERR_UNSUPPORTED, "3-D in-plane window %d has no kernel instance (1..15 odd)", p->k[2]);
  const Geo3DInfo& g = p->g3;
  k3.Z = (int)p->shape[0];
  k3.H = (int)p->shape[1];
  k3.W = (int)p->shape[2];
  k3.kz = p->k[0];
  k3.hz1 = (k3.kz - 1) / 2;
  k3.hz2 = k3.kz / 2;
  k3.sz = p->stride[0];
  k3.sy = p->stride[1];
  k3.sx = p->stride[2];
  k3.OZ = (int)p->oshape[0];
  k3.OY = (int)p->oshape[1];
  k3.OX = (int)p->oshape[2];
  k3.nyb = (k3.H + g.TY - 1) / g.TY;
  k3.nxb = (k3.W + g.TX - 1) / g.TX;
  k3.is_f32 = p->dtype == SWCORR_F32 ? 1 : 0;
  const uint64_t n = (uint64_t)p->k[0] * p->k[1] * p->k[2];
  k3.qbits = f32_qbits_3d(n, (uint64_t)p->k[1] * p->k[2]);
  if (!k3.is_f32 && (uint64_t)std::min(k3.kz, k3.Z) * std::min(p->k[1], k3.H) * std::min(p->k[2], k3.W) > kMaxU16Cells)
    return fail(SWCORR_ERR_UNSUPPORTED, "uint16 windows are limited to %llu in-bounds cells",
                (unsigned long long)kMaxU16Cells);
  const int eb = k3.is_f32 ? 4 : 2;
  const size_t slot = 2 * (((size_t)g.TYI * g.BXW * eb + 127) / 128 * 128);
  p->smem = 2 * slot + (size_t)8 * g.TY * g.VSP * 4 + 32;  // entering and leaving slot, vertical sums, barriers
  if (p->smem > (size_t)p->dev.smem_optin)
    return fail(SWCORR_ERR_UNSUPPORTED, "3-D plan needs %zu B of shared memory", p->smem);
  int per_sm = k3d_blocks_per_sm(p->k[2], p->smem);
  if (per_sm < 1) per_sm = 1;
  if (p->tune.ctas_per_sm > 0) per_sm = std::min(per_sm, p->tune.ctas_per_sm);
  const int slots = p->dev.sms * per_sm;
  const int planes_min = p->tune.tile_rows > 0 ? p->tune.tile_rows : 16;
  const int64_t F = (int64_t)k3.nyb * k3.nxb;
  int TZ = (int)std::min<int64_t>(k3.Z, std::max<int64_t>(planes_min, (k3.Z * F + 4 * slots - 1) / (4 * slots)));
  TZ = std::max(1, TZ);
  k3.TZ = TZ;
  k3.nzb = (k3.Z + TZ - 1) / TZ;
  k3.n_items = (int)(k3.nzb * F);
  k3.opy = k3.OX;
  k3.opz = (long long)k3.OY * k3.OX;
  p->grid = std::min(k3.n_items, slots);
  p->tune.prefetch = 2;
  p->tune.tile_rows = planes_min;
  p->tune.ctas_per_sm = per_sm;
  return SWCORR_OK;
}

static swcorr_status run_3d(swcorr_plan_s* p, const void* x, const void* y, const int64_t* in_pitch, float* c,
                            const int64_t* out_pitch, cudaStream_t st) {
  K3DParams& k3 = p->k3;
  const int eb = (int)elem_size(p->dtype);
  const int64_t py = in_pitch ? in_pitch[1] : k3.W;
  const int64_t pz = in_pitch ? in_pitch[0] : (int64_t)k3.H * py;
  if (in_pitch && in_pitch[2] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "in_pitch[2] must be 1");
  if (py < k3.W || pz < (int64_t)k3.H * py) return fail(SWCORR_ERR_INVALID_ARG, "input pitches too small");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (eb - 1))
    return fail(SWCORR_ERR_ALIGNMENT, "x and y must be aligned to their element size");
  // TMA needs 16-byte aligned bases and pitches; otherwise plain loads
  const bool tma =
      !(((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) || (py * eb) % 16 || (pz * eb) % 16);
  k3.use_tma = tma ? 1 : 0;
  k3.gx = x;
  k3.gy = y;
  k3.ipy = py;
  k3.ipz = pz;
  if (out_pitch) {
    if (out_pitch[2] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "out_pitch[2] must be 1");
    k3.opz = out_pitch[0];
    k3.opy = out_pitch[1];
  } else {
    k3.opy = k3.OX;
    k3.opz = (long long)k3.OY * k3.OX;
  }
  if (tma && (x != p->cached_x || y != p->cached_y || py != p->cached_pitch)) {
    const CUtensorMapDataType dt = p->dtype == SWCORR_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                          : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    swcorr_status s1 = encode_3d(&k3.tmx, dt, eb, x, k3.W, k3.H, k3.Z, py, pz, p->g3.BXW, p->g3.TYI);
    if (s1 == SWCORR_OK) s1 = encode_3d(&k3.tmy, dt, eb, y, k3.W, k3.H, k3.Z, py, pz, p->g3.BXW, p->g3.TYI);
    if (s1 != SWCORR_OK) {
      p->cached_x = p->cached_y = nullptr;
      return s1;
    }
    p->cached_x = x;
    p->cached_y = y;
    p->cached_pitch = py;
  }
  k3.out = c;
  k3.status = p->d_status;
  k3.unit_stride = (k3.sz == 1 && k3.sy == 1 && k3.sx == 1) ? 1 : 0;
  k3.vec_store = (k3.unit_stride && (reinterpret_cast<uintptr_t>(c) & 15) == 0 && k3.opy % 4 == 0 && k3.opz % 4 == 0)
                     ? 1 : 0;
  cudaError_t e;
  if (k3.is_f32) {
    // items the 22-bit map leaves uncertified go to the wide kernel
    k3.redo_count = p->d_redo;
    k3.redo_items = p->d_redo + 1;
    if ((e = cudaMemsetAsync(p->d_redo, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "3-D item list reset");
  } else {
    k3.redo_count = k3.redo_items = nullptr;
  }
  e = k3d_launch(p->k[2], k3, p->grid, p->smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "3-D kernel launch");
  if (k3.is_f32 && (e = k3d_wide_launch(p->k[2], k3, p->grid, p->smem, st)) != cudaSuccess)
    return cuda_fail(e, "3-D wide kernel launch");
  return SWCORR_OK;
}

// General n-D path: geometry; its buffers are allocated with the plan.
static swcorr_status plan_nd(swcorr_plan_s* p) {
  KNDParams& kn = p->kn;
  kn.ndim = p->ndim;
  int64_t cells = 1, outs = 1;
  uint64_t nmax = 1;
  for (int d = p->ndim - 1; d >= 0; d--) {
    kn.shape[d] = p->shape[d];
    kn.inner[d] = cells;
    kn.h1[d] = (p->k[d] - 1) / 2;
    kn.h2[d] = p->k[d] / 2;
    kn.stride[d] = p->stride[d];
    kn.oshape[d] = p->oshape[d];
    if ((double)cells * (double)p->shape[d] > 4.0e12)
      return fail(SWCORR_ERR_UNSUPPORTED, "grid too large for the general n-D path");
    cells *= p->shape[d];
    outs *= p->oshape[d];
    nmax *= (uint64_t)std::min<int64_t>(p->k[d], p->shape[d]);
  }
  kn.ncell = cells;
  kn.nout = outs;
  kn.paper = p->border == SWCORR_BORDER_PAPER ? 1 : 0;
  kn.sat = (p->flags & SWCORR_FLAG_SAT) ? 1 : 0;
  kn.nstreams = kn.paper ? 6 : 5;
  kn.is_f32 = p->dtype == SWCORR_F32 ? 1 : 0;
  if (!kn.is_f32 && nmax > (uint64_t)1 << 30)
    return fail(SWCORR_ERR_UNSUPPORTED, "uint16 windows of the n-D path are limited to 2^30 cells");
  // float32: |X| < 2^q per cell and n 2^(2q) < 2^62 keeps the window sums of
  // squares exact in int64; at most 22 bits (the rounding constant)
  int q = 22;
  while (q > 1 && std::ldexp((double)nmax, 2 * q) >= std::ldexp(1.0, 62)) q--;
  kn.qbits = q;
  return SWCORR_OK;
}

static swcorr_status run_nd(swcorr_plan_s* p, const void* x, const void* y, const int64_t* in_pitch, float* c,
                            const int64_t* out_pitch, int64_t* sums, cudaStream_t st) {
  KNDParams& kn = p->kn;
  const int64_t eb = (int64_t)elem_size(p->dtype);
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (eb - 1))
    return fail(SWCORR_ERR_ALIGNMENT, "x and y must be aligned to their element size");
  if (in_pitch) {
    if (in_pitch[p->ndim - 1] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "in_pitch[ndim-1] must be 1");
    for (int d = 0; d < p->ndim - 1; d++)
      if (in_pitch[d] < in_pitch[d + 1] * p->shape[d + 1])
        return fail(SWCORR_ERR_INVALID_ARG, "in_pitch[%d] too small", d);
  }
  if (out_pitch) {
    int64_t want = 1;
    for (int d = p->ndim - 1; d >= 0; d--) {
      if (out_pitch[d] != want) return fail(SWCORR_ERR_UNSUPPORTED, "the n-D path writes a contiguous output");
      want *= p->oshape[d];
    }
  }
  for (int d = 0; d < p->ndim; d++) kn.ipitch[d] = in_pitch ? in_pitch[d] : kn.inner[d];
  kn.x = x;
  kn.y = y;
  kn.out = c;
  kn.sums = reinterpret_cast<long long*>(sums);
  unsigned char* base = static_cast<unsigned char*>(p->d_nd);
  const size_t bytes = (size_t)kn.nstreams * (size_t)kn.ncell * 8;
  kn.buf[0] = reinterpret_cast<long long*>(base);
  kn.buf[1] = reinterpret_cast<long long*>(base + bytes);
  kn.scratch = reinterpret_cast<float*>(base + 2 * bytes);
  kn.segs = reinterpret_cast<long long*>(base + 2 * bytes + 64);
  kn.status = p->d_status;
  cudaError_t e = knd_launch(kn, p->dev.sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "n-D path launch");
  return SWCORR_OK;
}

static swcorr_status plan_2d(swcorr_plan_s* p) {
  swcorr_status st = setup_2d(p->dev, p->dtype, (int)p->shape[0], (int)p->shape[1], p->k[0], p->k[1],
                              p->stride[0], p->stride[1], &p->g2, &p->k2, &p->smem, &p->grid, &p->tune);
  p->k2.sc.test_stall = (p->flags & SWCORR_FLAG_TEST_STALL) ? 1 : 0;
  return st;
}

extern "C" {

const char* swcorr_status_string(swcorr_status s) {
  switch (s) {
    case SWCORR_OK: return "ok";
    case SWCORR_ERR_INVALID_ARG: return "invalid argument";
    case SWCORR_ERR_UNSUPPORTED: return "unsupported";
    case SWCORR_ERR_ALIGNMENT: return "alignment";
    case SWCORR_ERR_CUDA: return "CUDA error";
    case SWCORR_ERR_OOM: return "out of memory";
    case SWCORR_ERR_TIMEOUT: return "device wait timed out";
    case SWCORR_ERR_NO_DEVICE: return "no usable device";
  }
  return "unknown status";
}

const char* swcorr_last_error(void) { return g_last_error.c_str(); }

const char* swcorr_version(void) { return "swcorr 0.1.0 sm_103a"; }

swcorr_status swcorr_plan_create(swcorr_plan* out, int ndim, const int64_t* shape, const int32_t* k,
                                 const int32_t* stride, swcorr_dtype dtype, swcorr_border border, uint32_t flags) {
  return swcorr_plan_create_tuned(out, ndim, shape, k, stride, dtype, border, flags, nullptr);
}

swcorr_status swcorr_plan_tune(swcorr_plan p, swcorr_tune* out) {
  if (!p || !out) return fail(SWCORR_ERR_INVALID_ARG, "plan and out must not be NULL");
  *out = p->tune;
  return SWCORR_OK;
}

swcorr_status swcorr_plan_create_tuned(swcorr_plan* out, int ndim, const int64_t* shape, const int32_t* k,
                                       const int32_t* stride, swcorr_dtype dtype, swcorr_border border,
                                       uint32_t flags, const swcorr_tune* tune) {
  g_last_error.clear();
  if (!out) return fail(SWCORR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > KND_MAXDIM) return fail(SWCORR_ERR_UNSUPPORTED, "ndim must be 1 to 8 (got %d)", ndim);
  if (!shape || !k) return fail(SWCORR_ERR_INVALID_ARG, "shape and k must not be NULL");
  if (dtype != SWCORR_U16 && dtype != SWCORR_F32) return fail(SWCORR_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
  if (border != SWCORR_BORDER_CLIP && border != SWCORR_BORDER_PAPER)
    return fail(SWCORR_ERR_INVALID_ARG, "unknown border rule %d", (int)border);
  if (flags & ~(uint32_t)(SWCORR_FLAG_EMIT_SUMS | SWCORR_FLAG_TEST_STALL | SWCORR_FLAG_SAT | SWCORR_FLAG_UNFUSED))
    return fail(SWCORR_ERR_INVALID_ARG, "unknown flag bits 0x%x", flags);
  const bool general = ndim > 3 || (flags & (SWCORR_FLAG_SAT | SWCORR_FLAG_UNFUSED));
  if ((flags & SWCORR_FLAG_TEST_STALL) && general)
    return fail(SWCORR_ERR_INVALID_ARG, "SWCORR_FLAG_TEST_STALL applies to 2-D uint16 plans");
  if ((flags & SWCORR_FLAG_TEST_STALL) && !(ndim == 2 && dtype == SWCORR_U16))
    return fail(SWCORR_ERR_INVALID_ARG, "SWCORR_FLAG_TEST_STALL applies to 2-D uint16 plans");
  if ((flags & SWCORR_FLAG_EMIT_SUMS) && dtype != SWCORR_U16)
    return fail(SWCORR_ERR_INVALID_ARG, "SWCORR_FLAG_EMIT_SUMS needs uint16 data");
  if ((flags & SWCORR_FLAG_EMIT_SUMS) && border == SWCORR_BORDER_PAPER)
    return fail(SWCORR_ERR_INVALID_ARG, "SWCORR_FLAG_EMIT_SUMS applies to clipped windows");
  swcorr_plan_s tmp;
  tmp.ndim = ndim;
  tmp.dtype = dtype;
  tmp.flags = flags;
  tmp.border = border;
  for (int d = 0; d < ndim; d++) {
    if (shape[d] < 1) return fail(SWCORR_ERR_INVALID_ARG, "shape[%d] = %lld < 1", d, (long long)shape[d]);
    if (shape[d] > (1ll << 31) - 1024) return fail(SWCORR_ERR_UNSUPPORTED, "shape[%d] too large", d);
    if (k[d] < 1) return fail(SWCORR_ERR_INVALID_ARG, "k[%d] = %d < 1", d, k[d]);
    const int32_t s = stride ? stride[d] : 1;
    if (s < 1) return fail(SWCORR_ERR_INVALID_ARG, "stride[%d] = %d < 1", d, s);
    tmp.shape[d] = shape[d];
    tmp.k[d] = k[d];
    tmp.stride[d] = s;
    tmp.oshape[d] = (shape[d] + s - 1) / s;
  }
  swcorr_status st = tune_check(tune);
  if (st != SWCORR_OK) return st;
  st = device_info(&tmp.dev);
  if (st != SWCORR_OK) return st;
  if (tune) {
    tmp.tune = *tune;
  } else if (!tune_lookup(tmp.dev.name, "plain", ndim, tmp.k, dtype, &tmp.tune)) {
    tmp.tune = swcorr_tune{};
  }
  if (general) {
    tmp.kind = KIND_ND;
    st = plan_nd(&tmp);
  } else {
    if (ndim == 2) {
      tmp.kind = dtype == SWCORR_U16 ? KIND_2D_U16 : KIND_2D_F32;
      st = plan_2d(&tmp);
    } else if (ndim == 1) {
      tmp.kind = KIND_1D;
      st = plan_1d(&tmp);
    } else {
      tmp.kind = KIND_3D;
      st = plan_3d(&tmp);
    }
    // a window shape the fused kernel has no instance for (even or wide 2-D
    // widths, unequal or wide 3-D in-plane windows, very long 1-D windows,
    // uint16 windows beyond 32768 cells) runs on the general path
    if (st == SWCORR_ERR_UNSUPPORTED && !(flags & SWCORR_FLAG_TEST_STALL)) {
      g_last_error.clear();
      tmp.kind = KIND_ND;
      st = plan_nd(&tmp);
    } else if (st == SWCORR_OK && border == SWCORR_BORDER_PAPER) {
      // the fused kernel writes every window with clipped borders; a window
      // that neither passes an edge nor holds a missing value is whole, so
      // only the -2 outputs remain: the general path's mask-only pass
      swcorr_plan_s t2 = tmp;
      t2.kind = KIND_ND;
      st = plan_nd(&t2);
      if (st == SWCORR_OK && (t2.kn.nout >= (1ll << 31) || t2.kn.ncell >= (1ll << 31))) {
        // (the mask pass indexes in 32 bits): the general path instead
        tmp = t2;
      } else if (st == SWCORR_OK) {
        tmp.paper_post = true;
        tmp.kmask = t2.kn;
        tmp.kmask.mask_only = 1;
        tmp.kmask.nstreams = 1;
        tmp.kmask.sat = 0;
      }
    }
  }
  if (st != SWCORR_OK) return st;
  swcorr_plan_s* p = new (std::nothrow) swcorr_plan_s(tmp);
  if (!p) return fail(SWCORR_ERR_OOM, "host allocation of the plan failed");
  cudaError_t e = cudaMalloc(&p->d_status, ST_WORDS * sizeof(uint32_t));
  if (e != cudaSuccess) {
    delete p;
    return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "status block: out of device memory")
                                          : cuda_fail(e, "cudaMalloc(status)");
  }
  e = cudaMemset(p->d_status, 0, ST_WORDS * sizeof(uint32_t));
  if (e != cudaSuccess) {
    cudaFree(p->d_status);
    delete p;
    return cuda_fail(e, "cudaMemset(status)");
  }
  p->k2.status = p->d_status;
  if (p->paper_post) {
    // float32: two missing-count buffers (int64 per cell) and the scratch
    // words; uint16 holds no missing value and needs the scratch only
    const size_t bytes = p->dtype == SWCORR_F32 ? 2 * (size_t)p->kmask.ncell * 8 + 64 : 64;
    e = cudaMalloc(&p->d_mask, bytes);
    if (e != cudaSuccess) {
      swcorr_plan_destroy(p);
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "-2 mask buffers (%zu B): out of device memory", bytes)
                                            : cuda_fail(e, "cudaMalloc(-2 mask buffers)");
    }
  }
  if (p->kind == KIND_2D_F32) {
    // second-tier tasks of at most redo_rows output rows: every item can list
    // all of its rows once, so the list never fills
    Scene2D& sc = p->k2.sc;
    // (short windows: short tasks spread a few listed items over many warps;
    // tall windows: 2 kh rows keep the kh - 1 warm-up rows below half)
    sc.redo_rows = sc.kh <= 8 ? 8 : 2 * sc.kh;
    sc.redo_cap = p->k2.n_items * ((sc.TJ + sc.redo_rows - 1) / sc.redo_rows);
    e = cudaMalloc(&p->d_redo, 256 + (size_t)sc.redo_cap * sizeof(RedoTask2D) +
                                   (size_t)p->k2.n_items * 32 * sizeof(float4));
    if (e != cudaSuccess) {
      swcorr_plan_destroy(p);
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "2-D task list: out of device memory")
                                            : cuda_fail(e, "cudaMalloc(2-D task list)");
    }
    sc.redo_count = p->d_redo;
    sc.redo_tasks = reinterpret_cast<RedoTask2D*>(reinterpret_cast<unsigned char*>(p->d_redo) + 256);
    sc.redo_ranges = reinterpret_cast<float4*>(sc.redo_tasks + sc.redo_cap);
  }
  if (p->kind == KIND_1D && p->dtype == SWCORR_F32) {
    e = cudaMalloc(&p->d_redo, 8 + (size_t)p->k1.n_items * sizeof(long long));
    if (e != cudaSuccess) {
      swcorr_plan_destroy(p);
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "1-D chunk list: out of device memory")
                                            : cuda_fail(e, "cudaMalloc(1-D chunk list)");
    }
  }
  if (p->kind == KIND_3D && p->dtype == SWCORR_F32) {
    e = cudaMalloc(&p->d_redo, ((size_t)p->k3.n_items + 1) * sizeof(int));
    if (e != cudaSuccess) {
      swcorr_plan_destroy(p);
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "3-D item list: out of device memory")
                                            : cuda_fail(e, "cudaMalloc(3-D item list)");
    }
  }
  if (p->kind == KIND_ND) {
    // two stream buffers, scratch, and for the cumulative-sum ablation the
    // segment totals of the widest pass (at most ncell / 128 + lines per stream)
    size_t segs = 0;
    if (p->kn.sat)
      for (int d = 0; d < p->ndim - 1; d++)
        segs = std::max(segs, (size_t)((p->kn.ncell / p->kn.shape[d]) * ((p->kn.shape[d] + 127) / 128)));
    const size_t bytes = 2 * (size_t)p->kn.nstreams * (size_t)p->kn.ncell * 8 + 64 + (size_t)p->kn.nstreams * segs * 8;
    e = cudaMalloc(&p->d_nd, bytes);
    if (e != cudaSuccess) {
      swcorr_plan_destroy(p);
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "n-D stream buffers (%zu B): out of device memory", bytes)
                                            : cuda_fail(e, "cudaMalloc(n-D buffers)");
    }
  }
  *out = p;
  return SWCORR_OK;
}

int64_t swcorr_plan_outputs(swcorr_plan p) { return p ? n_outputs(p) : -1; }

static swcorr_status run_2d(swcorr_plan_s* p, const void* x, const void* y, const int64_t* in_pitch, float* c,
                            const int64_t* out_pitch, int64_t* sums, cudaStream_t st) {
  const int64_t W = p->shape[1];
  const int64_t ip = in_pitch ? in_pitch[0] : W;
  if (in_pitch && in_pitch[1] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "in_pitch[1] must be 1");
  if (ip < W) return fail(SWCORR_ERR_INVALID_ARG, "in_pitch[0] = %lld < cols = %lld", (long long)ip, (long long)W);
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & (elem_size(p->dtype) - 1))
    return fail(SWCORR_ERR_ALIGNMENT, "x and y must be aligned to their element size");
  const int64_t op = out_pitch ? out_pitch[0] : p->oshape[1];
  if (out_pitch && out_pitch[1] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "out_pitch[1] must be 1");
  if (op < p->oshape[1]) return fail(SWCORR_ERR_INVALID_ARG, "out_pitch[0] smaller than the output row");
  const bool cached = x == p->cached_x && y == p->cached_y && ip == p->cached_pitch;
  bool use_tma = false;
  swcorr_status s1 = bind_2d(&p->k2, p->g2, p->dtype, x, y, ip, c, op, sums, !cached, &use_tma);
  if (s1 != SWCORR_OK) {
    p->cached_x = p->cached_y = nullptr;
    return s1;
  }
  if (use_tma) {
    p->cached_x = x;
    p->cached_y = y;
    p->cached_pitch = ip;
  }
  cudaError_t e;
  if (p->dtype == SWCORR_F32 && p->d_redo) {
    // the items list their second tier; a second launch spreads its tasks
    // over every SM (it exits at once when nothing was listed)
    if ((e = cudaMemsetAsync(p->d_redo, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "2-D task list reset");
    if ((e = k2d_f32_launch(p->k2.sc.kw, p->k2, p->grid, p->smem, st, use_tma, 1)) != cudaSuccess)
      return cuda_fail(e, "2-D kernel launch");
    e = k2d_f32_launch(p->k2.sc.kw, p->k2, p->grid, p->smem, st, use_tma, 2);
  } else {
    e = p->dtype == SWCORR_F32 ? k2d_f32_launch(p->k2.sc.kw, p->k2, p->grid, p->smem, st, use_tma)
                               : k2d_u16_launch(p->k2.sc.kw, p->k2, p->grid, p->smem, st, use_tma);
  }
  if (e != cudaSuccess) return cuda_fail(e, "2-D kernel launch");
  return SWCORR_OK;
}

// The -2 outputs of the paper's convention after a fused run (knd.cu's
// mask-only form).
static swcorr_status run_mask(swcorr_plan_s* p, const void* x, const void* y, const int64_t* in_pitch, float* c,
                              cudaStream_t st) {
  KNDParams& km = p->kmask;
  if (in_pitch) {
    if (in_pitch[p->ndim - 1] != 1) return fail(SWCORR_ERR_UNSUPPORTED, "in_pitch[ndim-1] must be 1");
    for (int d = 0; d < p->ndim - 1; d++)
      if (in_pitch[d] < in_pitch[d + 1] * p->shape[d + 1])
        return fail(SWCORR_ERR_INVALID_ARG, "in_pitch[%d] too small", d);
  }
  for (int d = 0; d < p->ndim; d++) km.ipitch[d] = in_pitch ? in_pitch[d] : km.inner[d];
  km.x = x;
  km.y = y;
  km.out = c;
  km.sums = nullptr;
  unsigned char* base = static_cast<unsigned char*>(p->d_mask);
  const size_t bytes = p->dtype == SWCORR_F32 ? (size_t)km.ncell * 8 : 0;
  km.buf[0] = reinterpret_cast<long long*>(base);
  km.buf[1] = reinterpret_cast<long long*>(base + bytes);
  km.scratch = reinterpret_cast<float*>(base + 2 * bytes);
  km.segs = nullptr;
  km.status = p->d_status;
  cudaError_t e = knd_launch(km, p->dev.sms, st);
  if (e != cudaSuccess) return cuda_fail(e, "-2 mask launch");
  return SWCORR_OK;
}

swcorr_status swcorr_run(swcorr_plan p, const void* x, const void* y, const int64_t* in_pitch, float* c,
                         const int64_t* out_pitch, int64_t* sums, void* stream) {
  g_last_error.clear();
  if (!p) return fail(SWCORR_ERR_INVALID_ARG, "plan is NULL");
  if (p->kind == KIND_BATCHED) return fail(SWCORR_ERR_INVALID_ARG, "batched plans run with swcorr_run_batched");
  if (!x || !y || !c) return fail(SWCORR_ERR_INVALID_ARG, "x, y and c must not be NULL");
  if (reinterpret_cast<uintptr_t>(c) & 3) return fail(SWCORR_ERR_ALIGNMENT, "c must be 4-byte aligned");
  if (reinterpret_cast<uintptr_t>(sums) & 7) return fail(SWCORR_ERR_ALIGNMENT, "sums must be 8-byte aligned");
  if ((p->flags & SWCORR_FLAG_EMIT_SUMS) && !sums)
    return fail(SWCORR_ERR_INVALID_ARG, "plan has SWCORR_FLAG_EMIT_SUMS: sums must not be NULL");
  if (!(p->flags & SWCORR_FLAG_EMIT_SUMS)) sums = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (p->paper_post) {
    if (out_pitch) {
      int64_t want = 1;
      for (int d = p->ndim - 1; d >= 0; d--) {
        if (out_pitch[d] != want) return fail(SWCORR_ERR_UNSUPPORTED, "the -2 convention writes a contiguous output");
        want *= p->oshape[d];
      }
    }
    swcorr_status s0 = SWCORR_OK;
    switch (p->kind) {
      case KIND_2D_U16:
      case KIND_2D_F32: s0 = run_2d(p, x, y, in_pitch, c, out_pitch, nullptr, st); break;
      case KIND_3D: p->k3.sums = nullptr; s0 = run_3d(p, x, y, in_pitch, c, out_pitch, st); break;
      case KIND_1D:
        if ((in_pitch && in_pitch[0] != 1) || (out_pitch && out_pitch[0] != 1))
          return fail(SWCORR_ERR_UNSUPPORTED, "1-D series must be contiguous");
        p->k1.sums = nullptr;
        s0 = run_1d(p, x, y, c, st);
        break;
      default: return fail(SWCORR_ERR_UNSUPPORTED, "plan kind %d cannot run", p->kind);
    }
    if (s0 != SWCORR_OK) return s0;
    return run_mask(p, x, y, in_pitch, c, st);
  }
  switch (p->kind) {
    case KIND_ND: return run_nd(p, x, y, in_pitch, c, out_pitch, sums, st);
    case KIND_2D_U16:
    case KIND_2D_F32: return run_2d(p, x, y, in_pitch, c, out_pitch, sums, st);
    case KIND_3D:
      p->k3.sums = reinterpret_cast<long long*>(sums);
      return run_3d(p, x, y, in_pitch, c, out_pitch, st);
    case KIND_1D:
      if ((in_pitch && in_pitch[0] != 1) || (out_pitch && out_pitch[0] != 1))
        return fail(SWCORR_ERR_UNSUPPORTED, "1-D series must be contiguous");
      p->k1.sums = reinterpret_cast<long long*>(sums);
      return run_1d(p, x, y, c, st);
  }
  return fail(SWCORR_ERR_UNSUPPORTED, "plan kind %d cannot run", p->kind);
}

// Host run of a 2-D plan, pipelined over bands of row blocks: the input rows
// a band needs (its rows plus the window halo) are copied in order on one
// stream; each band's kernel launch waits only for its own input and runs on
// its own stream, so band kernels overlap each other and the copies; each
// band's output rows go back as soon as its kernel ends.  The work forks from
// and joins back to `origin`.
static swcorr_status enqueue_banded(swcorr_plan_s* p, const K2DParams& k2, const void* x, const void* y, float* c,
                                    float* c_dev, bool use_tma, const int* weights, int nb_max, cudaStream_t origin) {
  cudaError_t e;
  const Scene2D& sc = k2.sc;
  const int64_t W = p->shape[1], H = p->shape[0];
  const size_t eb = elem_size(p->dtype);
  const int64_t OW = p->oshape[1];
  if ((e = cudaEventRecord(p->he_start, origin)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(p->hs_in, p->he_start, 0)) != cudaSuccess)
    return cuda_fail(e, "order host run after the caller's stream");
  const int n_rb = sc.n_rb;
  const int nb = std::min(nb_max, n_rb);
  // band b covers row blocks [rbs[b], rbs[b + 1]): weights give the shares
  // (small first and last bands shorten the pipeline's fill and drain)
  int rbs[swcorr_plan_s::kMaxBands + 1];
  {
    int64_t tot = 0, acc = 0;
    for (int b = 0; b < nb; b++) tot += nb == nb_max ? weights[b] : 1;
    rbs[0] = 0;
    for (int b = 0; b < nb; b++) {
      acc += nb == nb_max ? weights[b] : 1;
      rbs[b + 1] = (int)((int64_t)n_rb * acc / tot);
    }
  }
  int64_t rows_in = 0;  // input rows copied so far
  bool used[swcorr_plan_s::kBands] = {};
  const unsigned char* hx = static_cast<const unsigned char*>(x);
  const unsigned char* hy = static_cast<const unsigned char*>(y);
  unsigned char* dx = static_cast<unsigned char*>(p->d_x);
  unsigned char* dy = static_cast<unsigned char*>(p->d_y);
  for (int b = 0; b < nb; b++) {
    const int rb0 = rbs[b], rb1 = rbs[b + 1];
    if (rb1 <= rb0) continue;
    const int64_t j1 = std::min<int64_t>((int64_t)rb1 * sc.TJ, sc.OH);  // output rows [rb0 TJ, j1)
    const int64_t need = std::min<int64_t>(H, (j1 - 1) * sc.sy + sc.h2 + 1);  // input rows the band reads
    if (need > rows_in) {
      const size_t off = (size_t)rows_in * W * eb, bytes = (size_t)(need - rows_in) * W * eb;
      if ((e = cudaMemcpyAsync(dx + off, hx + off, bytes, cudaMemcpyHostToDevice, p->hs_in)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dy + off, hy + off, bytes, cudaMemcpyHostToDevice, p->hs_in)) != cudaSuccess)
        return cuda_fail(e, "copy input band to device");
      rows_in = need;
    }
    cudaStream_t sk = p->hs_k[b % swcorr_plan_s::kBands];
    used[b % swcorr_plan_s::kBands] = true;
    if ((e = cudaEventRecord(p->he_in[b], p->hs_in)) != cudaSuccess || (e = cudaStreamWaitEvent(sk, p->he_in[b], 0)) != cudaSuccess)
      return cuda_fail(e, "band input event");
    K2DParams kp = k2;
    kp.rb0 = rb0;
    if (c_dev) {  // the band kernel stores straight into the caller's page-locked c
      kp.sc.out = c_dev;
      kp.sc.out_pitch = OW;
      kp.sc.vec_store = (sc.sx == 1 && (reinterpret_cast<uintptr_t>(c_dev) & 15) == 0 && (OW % 4) == 0) ? 1 : 0;
    }
    kp.n_items = (rb1 - rb0) * sc.n_strips;
    const int grid = std::min(kp.n_items, p->grid);
    e = p->dtype == SWCORR_F32 ? k2d_f32_launch(sc.kw, kp, grid, p->smem, sk, use_tma)
                               : k2d_u16_launch(sc.kw, kp, grid, p->smem, sk, use_tma);
    if (e != cudaSuccess) return cuda_fail(e, "2-D band kernel launch");
    if ((e = cudaEventRecord(p->he_k[b], sk)) != cudaSuccess || (e = cudaStreamWaitEvent(p->hs_out, p->he_k[b], 0)) != cudaSuccess)
      return cuda_fail(e, "band kernel event");
    if (c_dev) continue;
    const int64_t o0 = (int64_t)rb0 * sc.TJ;
    const size_t ooff = (size_t)o0 * OW * sizeof(float), obytes = (size_t)(j1 - o0) * OW * sizeof(float);
    if ((e = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(c) + ooff,
                             reinterpret_cast<unsigned char*>(p->d_c) + ooff, obytes, cudaMemcpyDeviceToHost,
                             p->hs_out)) != cudaSuccess)
      return cuda_fail(e, "copy output band to host");
  }
  // join every forked stream back to the origin
  if ((e = cudaEventRecord(p->he_done, p->hs_out)) != cudaSuccess || (e = cudaStreamWaitEvent(origin, p->he_done, 0)) != cudaSuccess ||
      (e = cudaEventRecord(p->he_in[0], p->hs_in)) != cudaSuccess || (e = cudaStreamWaitEvent(origin, p->he_in[0], 0)) != cudaSuccess)
    return cuda_fail(e, "join host run");
  for (int b = 0; b < swcorr_plan_s::kBands; b++)
    if (used[b] && ((e = cudaEventRecord(p->he_k[b], p->hs_k[b])) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(origin, p->he_k[b], 0)) != cudaSuccess))
      return cuda_fail(e, "join host run");
  return SWCORR_OK;
}

// Band shares of the recorded pipeline: small first and last bands shorten
// the fill (input copy of the first band, alone) and the tail (the last
// band's kernel and its output, alone); the middle bands overlap both
// directions of the host link.
static const int kGraphBandWeights[swcorr_plan_s::kGraphBands] = {1, 4, 6, 4, 1};
static const int kStreamBandWeights[swcorr_plan_s::kBands] = {1, 1, 1, 1, 1, 1, 1, 1};

static bool page_locked(const void* ptr, void** dev_alias = nullptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (dev_alias) *dev_alias = a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  return a.type == cudaMemoryTypeHost;
}

// Band kernels of the recorded host run write c through its device mapping
// (no separate output copies); the results then stream back over the host
// link while later bands compute and their inputs arrive.
static constexpr bool kDirectHostOutput = true;

// Synchronous, like swcorr_run_host.  With page-locked x, y and c the band
// pipeline is recorded once as a CUDA graph (keyed by the three pointers)
// and replayed with one launch, so the host issues one call instead of about
// ten per band; pageable buffers take the stream path.
static swcorr_status run_host_2d_banded(swcorr_plan_s* p, const void* x, const void* y, float* c, cudaStream_t st) {
  cudaError_t e;
  if (!p->hs_in) {
    bool ok = cudaStreamCreateWithFlags(&p->hs_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->hs_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->hs_cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->he_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->he_done, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; ok && b < swcorr_plan_s::kBands; b++)
      ok = cudaStreamCreateWithFlags(&p->hs_k[b], cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < swcorr_plan_s::kMaxBands; b++)
      ok = cudaEventCreateWithFlags(&p->he_in[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&p->he_k[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_fail(cudaGetLastError(), "host-run streams and events");
  }
  const int64_t W = p->shape[1];
  const int64_t OW = p->oshape[1];
  // bind the staging buffers once (tensor maps of the whole staged image)
  const bool cached = p->d_x == p->cached_x && p->d_y == p->cached_y && W == p->cached_pitch;
  bool use_tma = false;
  swcorr_status s1 = bind_2d(&p->k2, p->g2, p->dtype, p->d_x, p->d_y, W, p->d_c, OW, nullptr, !cached, &use_tma);
  if (s1 != SWCORR_OK) {
    p->cached_x = p->cached_y = nullptr;
    return s1;
  }
  if (use_tma) {
    p->cached_x = p->d_x;
    p->cached_y = p->d_y;
    p->cached_pitch = W;
  }
  bool graphed = false;
  void* c_alias = nullptr;
  if (page_locked(x) && page_locked(y) && page_locked(c, &c_alias)) {
    float* c_dev = kDirectHostOutput ? static_cast<float*>(c_alias) : nullptr;
    if (!p->hgraph_exec || p->hg_x != x || p->hg_y != y || p->hg_c != c || p->hg_tma != use_tma) {
      if (p->hgraph_exec) cudaGraphExecDestroy(p->hgraph_exec);
      p->hgraph_exec = nullptr;
      // record; if anything in the recording fails, the stream path below
      // runs instead (and reports a real error itself)
      if (cudaStreamBeginCapture(p->hs_cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        swcorr_status s2 =
            enqueue_banded(p, p->k2, x, y, c, c_dev, use_tma, kGraphBandWeights, swcorr_plan_s::kGraphBands, p->hs_cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->hs_cap, &g);
        if (s2 == SWCORR_OK && e == cudaSuccess && g && cudaGraphInstantiate(&p->hgraph_exec, g, 0) != cudaSuccess)
          p->hgraph_exec = nullptr;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
      g_last_error.clear();
      p->hg_x = x;
      p->hg_y = y;
      p->hg_c = c;
      p->hg_tma = use_tma;
    }
    if (p->hgraph_exec) {
      if ((e = cudaGraphLaunch(p->hgraph_exec, st)) != cudaSuccess) return cuda_fail(e, "launch host-run graph");
      graphed = true;
    }
  }
  if (!graphed) {
    swcorr_status s2 = enqueue_banded(p, p->k2, x, y, c, nullptr, use_tma, kStreamBandWeights, swcorr_plan_s::kBands, st);
    if (s2 != SWCORR_OK) {
      // nothing queued so far may still touch the caller's buffers on return
      const std::string msg = g_last_error;
      cudaStreamSynchronize(p->hs_in);
      for (int b = 0; b < swcorr_plan_s::kBands; b++) cudaStreamSynchronize(p->hs_k[b]);
      cudaStreamSynchronize(p->hs_out);
      cudaGetLastError();
      g_last_error = msg;
      return s2;
    }
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "host run synchronize");
  return SWCORR_OK;
}

swcorr_status swcorr_run_host(swcorr_plan p, const void* x, const void* y, float* c, void* stream) {
  g_last_error.clear();
  if (!p) return fail(SWCORR_ERR_INVALID_ARG, "plan is NULL");
  if (!x || !y || !c) return fail(SWCORR_ERR_INVALID_ARG, "x, y and c must not be NULL");
  if (p->kind == KIND_BATCHED) return fail(SWCORR_ERR_INVALID_ARG, "batched plans have no host run");
  if (p->flags & SWCORR_FLAG_EMIT_SUMS) return fail(SWCORR_ERR_INVALID_ARG, "host runs do not emit sums");
  int64_t nin = 1;
  for (int d = 0; d < p->ndim; d++) nin *= p->shape[d];
  const size_t in_bytes = (size_t)nin * elem_size(p->dtype);
  const size_t out_bytes = (size_t)n_outputs(p) * sizeof(float);
  cudaError_t e;
  if (!p->d_x) {
    // rows padded to 16 bytes so the device copy satisfies the TMA pitch rule
    if ((e = cudaMalloc(&p->d_x, in_bytes + 64)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_y, in_bytes + 64)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_c, out_bytes + 64)) != cudaSuccess) {
      cudaFree(p->d_x);
      cudaFree(p->d_y);
      cudaFree(p->d_c);
      p->d_x = p->d_y = nullptr;
      p->d_c = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "staging buffers: out of device memory")
                                            : cuda_fail(e, "cudaMalloc(staging)");
    }
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t inner = p->shape[p->ndim - 1];
  if (p->kind != KIND_ND && p->ndim >= 2 && (inner * (int64_t)elem_size(p->dtype)) % 16 != 0)
    return fail(SWCORR_ERR_ALIGNMENT, "host runs need rows of a multiple of 16 bytes (got %lld elements)",
                (long long)inner);
  if ((p->kind == KIND_2D_U16 || p->kind == KIND_2D_F32) && !p->paper_post) return run_host_2d_banded(p, x, y, c, st);
  if ((e = cudaMemcpyAsync(p->d_x, x, in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "copy x to device");
  if ((e = cudaMemcpyAsync(p->d_y, y, in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "copy y to device");
  swcorr_status s = swcorr_run(p, p->d_x, p->d_y, nullptr, p->d_c, nullptr, nullptr, stream);
  if (s != SWCORR_OK) return s;
  if ((e = cudaMemcpyAsync(c, p->d_c, out_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy c to host");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return SWCORR_OK;
}

swcorr_status swcorr_plan_status(swcorr_plan p) {
  g_last_error.clear();
  if (!p) return fail(SWCORR_ERR_INVALID_ARG, "plan is NULL");
  uint32_t h[ST_WORDS];
  cudaError_t e = cudaMemcpy(h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status block");
  uint32_t zero = 0;
  cudaMemcpy(p->d_status + ST_ERROR, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (h[ST_ERROR] & ERRBIT_TIMEOUT) return fail(SWCORR_ERR_TIMEOUT, "a kernel's bounded wait gave up");
  if (h[ST_ERROR]) return fail(SWCORR_ERR_CUDA, "device status bits 0x%x", h[ST_ERROR]);
  return SWCORR_OK;
}

int64_t swcorr_plan_fallbacks(swcorr_plan p) {
  if (!p) return -1;
  uint32_t v = 0;
  if (cudaMemcpy(&v, p->d_status + ST_FALLBACK, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  uint32_t zero = 0;
  cudaMemcpy(p->d_status + ST_FALLBACK, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  return v;
}

void swcorr_plan_destroy(swcorr_plan p) {
  if (!p) return;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_batch);
  cudaFree(p->d_nd);
  cudaFree(p->d_mask);
  cudaFree(p->d_redo);
  cudaFree(p->d_status);
  cudaFree(p->d_x);
  cudaFree(p->d_y);
  cudaFree(p->d_c);
  if (p->hgraph_exec) cudaGraphExecDestroy(p->hgraph_exec);
  if (p->hs_in) cudaStreamDestroy(p->hs_in);
  if (p->hs_out) cudaStreamDestroy(p->hs_out);
  if (p->hs_cap) cudaStreamDestroy(p->hs_cap);
  if (p->he_start) cudaEventDestroy(p->he_start);
  if (p->he_done) cudaEventDestroy(p->he_done);
  for (int b = 0; b < swcorr_plan_s::kBands; b++)
    if (p->hs_k[b]) cudaStreamDestroy(p->hs_k[b]);
  for (int b = 0; b < swcorr_plan_s::kMaxBands; b++) {
    if (p->he_in[b]) cudaEventDestroy(p->he_in[b]);
    if (p->he_k[b]) cudaEventDestroy(p->he_k[b]);
  }
  delete p;
}

swcorr_status swcorr_plan_batched(swcorr_plan* out, const swcorr_scene* scenes, int n_scenes, swcorr_dtype dtype,
                                  uint32_t flags) {
  return swcorr_plan_batched_tuned(out, scenes, n_scenes, dtype, flags, nullptr);
}

swcorr_status swcorr_plan_batched_tuned(swcorr_plan* out, const swcorr_scene* scenes, int n_scenes,
                                        swcorr_dtype dtype, uint32_t flags, const swcorr_tune* tune) {
  g_last_error.clear();
  if (!out) return fail(SWCORR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!scenes || n_scenes < 1) return fail(SWCORR_ERR_INVALID_ARG, "need at least one scene");
  if (dtype != SWCORR_U16 && dtype != SWCORR_F32) return fail(SWCORR_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
  const bool f32 = dtype == SWCORR_F32;
  if (flags != 0) return fail(SWCORR_ERR_INVALID_ARG, "batched plans take no flags");
  swcorr_status st = tune_check(tune);
  if (st != SWCORR_OK) return st;
  DeviceInfo dev;
  st = device_info(&dev);
  if (st != SWCORR_OK) return st;
  swcorr_tune tn{};
  if (tune) {
    tn = *tune;
  } else if (!tune_lookup(dev.name, "batched", 2, nullptr, dtype, &tn)) {
    tn = swcorr_tune{};
  }
  // least output rows per work item (float32: taller items amortise the
  // second tier's halo rows; 128 measured best on mixed scenes)
  const int rows_min = tn.tile_rows > 0 ? tn.tile_rows : (f32 ? 128 : 64);
  cudaError_t e = f32 ? kbatched_f32_prepare() : kbatched_prepare();
  if (e != cudaSuccess) return cuda_fail(e, "batched kernel attributes");

  // per-scene set-up on the host
  std::vector<Scene2D> sc(n_scenes);
  std::vector<CUtensorMap> maps(4 * (size_t)n_scenes);
  std::vector<double> cost(n_scenes);
  int64_t outputs = 0;
  for (int i = 0; i < n_scenes; i++) {
    const swcorr_scene& s = scenes[i];
    if (s.shape[0] < 1 || s.shape[1] < 1 || s.shape[0] > (1ll << 31) - 1024 || s.shape[1] > (1ll << 31) - 1024)
      return fail(SWCORR_ERR_INVALID_ARG, "scene %d: bad shape", i);
    if (s.k[0] < 1 || s.k[1] < 1) return fail(SWCORR_ERR_INVALID_ARG, "scene %d: bad window", i);
    if (!f32 && (uint64_t)std::min<int64_t>(s.k[0], s.shape[0]) * (uint64_t)std::min<int64_t>(s.k[1], s.shape[1]) > kMaxU16Cells)
      return fail(SWCORR_ERR_UNSUPPORTED, "scene %d: uint16 windows are limited to %llu in-bounds cells", i,
                  (unsigned long long)kMaxU16Cells);
    Geo2DInfo g;
    if (!(f32 ? k2d_f32_geometry(s.k[1], &g) : k2d_u16_geometry(s.k[1], &g)) || g.M != 8)
      return fail(SWCORR_ERR_UNSUPPORTED, "scene %d: window width %d has no kernel instance (1..31 odd)", i, s.k[1]);
    if (!s.x || !s.y || !s.c) return fail(SWCORR_ERR_INVALID_ARG, "scene %d: NULL pointer", i);
    if (s.in_pitch < s.shape[1] || s.out_pitch < s.shape[1])
      return fail(SWCORR_ERR_INVALID_ARG, "scene %d: pitch smaller than the row", i);
    if (((reinterpret_cast<uintptr_t>(s.x) | reinterpret_cast<uintptr_t>(s.y)) & 15) || (s.in_pitch * (f32 ? 4 : 2)) % 16)
      return fail(SWCORR_ERR_ALIGNMENT, "scene %d: batched inputs need 16-byte aligned bases and row pitches", i);
    Scene2D& q = sc[i];
    q.H = (int)s.shape[0];
    q.W = (int)s.shape[1];
    q.kh = s.k[0];
    q.h1 = (q.kh - 1) / 2;
    q.h2 = q.kh / 2;
    q.kw = s.k[1];
    q.sy = q.sx = 1;
    q.OH = q.H;
    q.OW = q.W;
    q.n_strips = (q.W + 32 * g.M - 1) / (32 * g.M);
    q.TJ = std::min(q.OH, std::max(rows_min, 2 * q.kh));  // the kh - 1 halo rows re-read stay below half
    q.n_rb = (q.OH + q.TJ - 1) / q.TJ;
    const uint64_t n = (uint64_t)q.kh * (uint64_t)q.kw;
    q.inv_n = n <= 1 ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / n);
    q.gx = s.x;
    q.gy = s.y;
    q.in_pitch = s.in_pitch;
    q.out = s.c;
    q.out_pitch = s.out_pitch;
    q.sums = nullptr;
    q.vec_store = ((reinterpret_cast<uintptr_t>(s.c) & 15) == 0 && (s.out_pitch % 4) == 0) ? 1 : 0;
    q.wide = (!f32 && (n > 64 || q.kw > 9)) ? 1 : 0;  // the batched kernel has 32-bit bodies for kw <= 9 only
    q.qbits = f32_qbits(n);
    const CUtensorMapDataType tdt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const int eb = f32 ? 4 : 2;
    st = encode_2d(&maps[4 * i + 0], tdt, eb, s.x, q.W, q.H, s.in_pitch, 256);
    if (st == SWCORR_OK) st = encode_2d(&maps[4 * i + 1], tdt, eb, s.y, q.W, q.H, s.in_pitch, 256);
    if (st == SWCORR_OK && g.TAIL > 0) {
      st = encode_2d(&maps[4 * i + 2], tdt, eb, s.x, q.W, q.H, s.in_pitch, g.TAIL);
      if (st == SWCORR_OK) st = encode_2d(&maps[4 * i + 3], tdt, eb, s.y, q.W, q.H, s.in_pitch, g.TAIL);
    }
    if (st != SWCORR_OK) return st;
    cost[i] = (double)(q.TJ + q.kh - 1) * (8 + q.kw - 1 + 16);
    outputs += (int64_t)q.H * q.W;
  }
  // work items, scenes with the costliest items first
  std::vector<int> order(n_scenes);
  for (int i = 0; i < n_scenes; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  // items grouped by kernel class (32-bit engine; 64-bit up to 17 columns;
  // 64-bit above), one launch each
  // (float32: one class per window width, so that each kernel holds the
  // registers of its own body only)
  const int n_cls = f32 ? kMaxBatchClasses : 3;
  auto cls_of = [&](int i) {
    if (f32) return (sc[i].kw - 1) / 2;
    return sc[i].wide == 0 ? 0 : (sc[i].kw <= 17 ? 1 : 2);
  };
  std::vector<BatchItem> items;
  size_t cls_start[kMaxBatchClasses + 1] = {};
  for (int cls = 0; cls < n_cls; cls++) {
    cls_start[cls] = items.size();
    for (int i : order) {
      if (cls_of(i) != cls) continue;
      for (int rb = 0; rb < sc[i].n_rb; rb++)
        for (int strip = 0; strip < sc[i].n_strips; strip++) items.push_back(BatchItem{i, strip, rb, 0});
    }
  }
  cls_start[n_cls] = items.size();
  if (items.size() > (size_t)0x7fffffff) return fail(SWCORR_ERR_UNSUPPORTED, "too many work items");

  // one device block: maps (64-byte aligned), scenes, items, counter
  const size_t maps_bytes = maps.size() * sizeof(CUtensorMap);
  const size_t sc_off = (maps_bytes + 255) / 256 * 256;
  const size_t it_off = sc_off + (n_scenes * sizeof(Scene2D) + 255) / 256 * 256;
  const size_t ctr_off = it_off + (items.size() * sizeof(BatchItem) + 255) / 256 * 256;
  const size_t total = ctr_off + 256;
  swcorr_plan_s* p = new (std::nothrow) swcorr_plan_s();
  if (!p) return fail(SWCORR_ERR_OOM, "host allocation of the plan failed");
  p->kind = KIND_BATCHED;
  p->ndim = 2;
  p->dtype = dtype;
  p->dev = dev;
  p->batched_outputs = outputs;
  p->n_cls = n_cls;
  auto cleanup = [&](swcorr_status s) {
    swcorr_plan_destroy(p);
    return s;
  };
  if ((e = cudaMalloc(&p->d_batch, total)) != cudaSuccess)
    return cleanup(e == cudaErrorMemoryAllocation ? fail(SWCORR_ERR_OOM, "batched plan: out of device memory")
                                                  : cuda_fail(e, "cudaMalloc(batched plan)"));
  if ((e = cudaMalloc(&p->d_status, ST_WORDS * sizeof(uint32_t))) != cudaSuccess)
    return cleanup(cuda_fail(e, "cudaMalloc(status)"));
  unsigned char* base = static_cast<unsigned char*>(p->d_batch);
  for (int i = 0; i < n_scenes; i++) {
    sc[i].tmx = reinterpret_cast<const CUtensorMap*>(base) + 4 * i + 0;
    sc[i].tmy = reinterpret_cast<const CUtensorMap*>(base) + 4 * i + 1;
    sc[i].tmx_t = reinterpret_cast<const CUtensorMap*>(base) + 4 * i + 2;
    sc[i].tmy_t = reinterpret_cast<const CUtensorMap*>(base) + 4 * i + 3;
  }
  if ((e = cudaMemcpy(base, maps.data(), maps_bytes, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(base + sc_off, sc.data(), n_scenes * sizeof(Scene2D), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(base + it_off, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemset(base + ctr_off, 0, 256)) != cudaSuccess ||
      (e = cudaMemset(p->d_status, 0, ST_WORDS * sizeof(uint32_t))) != cudaSuccess)
    return cleanup(cuda_fail(e, "batched plan upload"));
  const int PF = tn.prefetch > 0 ? tn.prefetch : (f32 ? 3 : 4);  // (float32: as the plain kernel)
  p->smem = f32 ? (size_t)4 * (PF + 1) * kbatched_f32_ring_row() * 4 + (size_t)(PF + 1) * 8
                : (size_t)4 * (PF + 1) * kbatched_ring_row() * 2 + (size_t)(PF + 1) * 8;
  int per_sm_max = 0;
  for (int cls = 0; cls < n_cls; cls++) {
    KBatchParams& kb = p->kbs[cls];
    kb.scenes = reinterpret_cast<const Scene2D*>(base + sc_off);
    kb.items = reinterpret_cast<const BatchItem*>(base + it_off) + cls_start[cls];
    kb.n_items = (int)(cls_start[cls + 1] - cls_start[cls]);
    kb.PF = PF;
    kb.NR = PF + 1;
    kb.counter = reinterpret_cast<uint32_t*>(base + ctr_off) + cls;
    kb.status = p->d_status;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f32 ? kbatched_f32_kernel_ptr(cls) : kbatched_kernel_ptr(cls),
                                                      32, p->smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 8;
    if (tn.ctas_per_sm > 0) per_sm = std::min(per_sm, tn.ctas_per_sm);
    p->bgrid[cls] = (int)std::min<int64_t>((int64_t)dev.sms * per_sm, kb.n_items);
    per_sm_max = std::max(per_sm_max, per_sm);
  }
  p->tune.prefetch = PF;
  p->tune.tile_rows = rows_min;
  p->tune.ctas_per_sm = per_sm_max;
  *out = p;
  return SWCORR_OK;
}

swcorr_status swcorr_run_batched(swcorr_plan p, void* stream) {
  g_last_error.clear();
  if (!p) return fail(SWCORR_ERR_INVALID_ARG, "plan is NULL");
  if (p->kind != KIND_BATCHED) return fail(SWCORR_ERR_INVALID_ARG, "not a batched plan");
  cudaError_t e;
  if (!p->graph_exec) {
    // capture {reset the work-queue counter; persistent kernel} once
    if ((e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "create capture stream");
    if ((e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "begin capture");
    cudaError_t e1 = cudaMemsetAsync(p->kbs[0].counter, 0, (size_t)p->n_cls * sizeof(uint32_t), p->cap_stream);
    // one launch per class with items, in sequence (concurrent branches let
    // the classes' CTAs share the SMs, which measured slower)
    cudaError_t e2 = e1;
    for (int cls = 0; cls < p->n_cls && e2 == cudaSuccess; cls++)
      if (p->kbs[cls].n_items > 0)
        e2 = p->dtype == SWCORR_F32 ? kbatched_f32_launch(p->kbs[cls], cls, p->bgrid[cls], p->smem, p->cap_stream)
                                    : kbatched_launch(p->kbs[cls], cls, p->bgrid[cls], p->smem, p->cap_stream);
    e = cudaStreamEndCapture(p->cap_stream, &p->graph);
    if (e1 != cudaSuccess) return cuda_fail(e1, "capture counter reset");
    if (e2 != cudaSuccess) return cuda_fail(e2, "capture batched kernel");
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    if ((e = cudaGraphInstantiate(&p->graph_exec, p->graph, 0)) != cudaSuccess) {
      p->graph_exec = nullptr;
      return cuda_fail(e, "instantiate graph");
    }
  }
  if ((e = cudaGraphLaunch(p->graph_exec, reinterpret_cast<cudaStream_t>(stream))) != cudaSuccess)
    return cuda_fail(e, "graph launch");
  return SWCORR_OK;
}

}  // extern "C"
