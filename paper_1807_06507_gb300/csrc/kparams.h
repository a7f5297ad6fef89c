// kparams.h -- parameter blocks shared by the host plan code and the kernels.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace swc {

// Device status block owned by each plan (uint32 words).
enum : int {
  ST_ERROR = 0,      // OR of ERRBIT_* below
  ST_FALLBACK = 1,   // windows recomputed by the exact per-window fallback
  ST_WORDS = 8
};
enum : uint32_t { ERRBIT_TIMEOUT = 1u, ERRBIT_BAD_ARG = 2u };


// A float32 2-D second-tier task: the lanes `lanes` of column strip `strip`
// re-march output rows [j0, j1) with a finer map (k2d_f32.cuh) of the value
// ranges their item measured, kept at redo_ranges[32 * range_slot + lane]
// (range_slot: the item's index).
struct RedoTask2D {
  int strip;
  int j0, j1;
  uint32_t lanes;
  int range_slot;
  int pad[3];
};

// One 2-D problem as the 2-D kernels see it.  All coordinates are input
// cells; output (j_r, j_c) has centre (j_r * sy, j_c * sx).
struct Scene2D {
  const CUtensorMap* tmx;  // tensor maps (param or global space, 64-byte aligned):
  const CUtensorMap* tmy;  //   boxes of 256 x 1 elements
  const CUtensorMap* tmx_t;//   and the tail box of a row span
  const CUtensorMap* tmy_t;
  int H, W;                // input rows, cols
  int kh, h1, h2;          // window rows and its extents above/below the centre
  int kw;                  // window cols (the kernel's compile-time KW must equal it)
  int sy, sx;              // strides
  int OH, OW;              // output rows, cols
  int TJ;                  // output rows per work item
  int n_strips;            // column strips of 32*M centre columns
  int n_rb;                // row blocks of TJ output rows
  uint32_t inv_n;          // floor(2^32 / (kh*kw)): mean estimate for interior windows
  int vec_store;           // 1: c rows are 16-byte aligned and sx == 1
  const void* gx;          // base pointers and row pitch (elements) for the
  const void* gy;          //   plain-load row loader (pitches TMA cannot take)
  long long in_pitch;
  float* out;
  long long out_pitch;     // elements between output rows
  long long* sums;         // optional 5 int64 per output (debug / bit-exact tests)
  int qbits;               // float32 path: fixed-point magnitude bits (|X| < 2^qbits)
  int wide;                // uint16 path: 64-bit second-moment sums (large windows)
  int test_stall;          // test hook: item (0, 0) never issues its first row's copy
  // float32 second tier listed as tasks of at most redo_rows output rows
  // (redo_tasks, redo_count, capacity redo_cap) for the launch that follows
  int redo_rows;
  int redo_cap;
  RedoTask2D* redo_tasks;
  int* redo_count;
  float4* redo_ranges;     // (lo_x, hi_x, lo_y, hi_y) per item and lane
};

struct K2DParams {
  CUtensorMap tmx;  // 64-byte aligned members first
  CUtensorMap tmy;
  CUtensorMap tmx_t;
  CUtensorMap tmy_t;
  Scene2D sc;
  int n_items;      // work items of this launch: row blocks [rb0, rb0 + n_items / n_strips) x strips
  int rb0;          // first row block (0 unless a launch covers one band of the output)
  int NR;           // ring rows
  int PF;           // rows prefetched ahead
  uint32_t* status;
};

// Batched: one persistent launch over many 2-D scenes.
struct BatchItem {
  int scene;
  int strip;
  int rb;
  int pad;
};

struct KBatchParams {
  const Scene2D* scenes;     // device array
  const BatchItem* items;    // device array, largest cost first
  int n_items;
  int NR, PF;
  uint32_t* counter;         // work-queue head (reset before every launch)
  uint32_t* status;
};

}  // namespace swc
