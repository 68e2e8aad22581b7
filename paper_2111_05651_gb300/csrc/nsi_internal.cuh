// Internal declarations of libnsi_assemble: the handle, status helpers and the
// per-element arithmetic shared by the kernels.  Nothing here is part of the
// public ABI (include/nsi_assemble.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nsi_assemble.h"

namespace nsi {

// ---------------------------------------------------------------- status ---
void set_error(const std::string& msg);
nsi_status fail(nsi_status s, const std::string& msg);
nsi_status cuda_fail(cudaError_t e, const char* what);

#define NSI_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return nsi::cuda_fail(e_, #call); \
  } while (0)

// device error word bits (set by kernels built with debug checks)
enum : unsigned { ERR_BAD_INDEX = 1u, ERR_NOT_IN_PATTERN = 2u, ERR_STAR = 4u };

// Row-gather ("pull") map, built at create time: for CSR row i, one 16-bit
// word per element that contains node i (the row's star): the positions,
// inside row i's column list, of the element's other three nodes (5 bits
// each), ordered so that (i, j1, j2, j3) is an even permutation of the
// element's node order (hence a positively oriented tet).  The kernels read
// the element walk encoded from these words (WALK_* below) and the edge-fan
// map.  Rows longer than 32 entries cannot be encoded; such meshes do not
// support the gather mode.
constexpr int STAR_BITS = 5;
constexpr int STAR_MAX_ROW = 1 << STAR_BITS;
// an element with |d1||d2||d3| > EXACT_RATIO |det| (edge vectors from any of
// its nodes) is "badly shaped": in the mixed modes the rows of its nodes are
// recomputed in double after the assembly
constexpr double EXACT_RATIO = 16.0;
// One step of a row's element walk (one byte): the row position of the node
// it brings into the window, whether the element formed by the window and that
// node is evaluated, the element's orientation in window order, and which
// window node leaves afterwards.
constexpr unsigned WALK_POS = 31u;       // bits 0-4: row position of the new node
constexpr unsigned WALK_ELEM = 1u << 5;  // the step evaluates element (p, q, c)
constexpr unsigned WALK_NEG = 1u << 6;   // (p, q, c) is an odd permutation of the element's order
constexpr unsigned WALK_EVQ = 1u << 7;   // q leaves (next window (p, c)); else p leaves (next window (q, c))

// Element-position map, for the element-centric kernels: per element one
// 64-bit word holding, for every ordered pair (a, b) of its local nodes with
// b != a, the position of node b inside the CSR row of node a, 5 bits each,
// at bit 5 * (3a + (b < a ? b : b - 1)); the diagonal positions come from
// diag_pos.  Built for meshes whose rows have at most 32 entries (others scan
// the row).
constexpr int ELEM_POS_BITS = 5;
__host__ __device__ inline int elem_pos_slot(int a, int b) { return 3 * a + (b < a ? b : b - 1); }

// Edge-fan map: for every off-diagonal CSR entry (i, j), the ring of nodes
// around the edge (i, j) -- the other two nodes of every element containing
// both i and j, chained in cyclic order so that consecutive ring nodes k, l
// form the positively oriented element (i, j, k, l) -- as positions inside
// row i.  One 32-bit word per entry: ring positions in bits 0..23 (4 bits
// each, up to 6 of them), ring size in bits 24..26, bit 27 set when the ring
// is closed (interior edge: as many elements as ring nodes) and clear when it
// is open (boundary edge: one element fewer).  The diagonal entry has word 0.
// Meshes with rows longer than 16 entries, rings longer than 6 nodes or
// non-manifold edge fans do not get the map and use the per-row star kernel.
constexpr int FAN_MAX_ROW = 16;
constexpr int FAN_MAX_RING = 6;
constexpr int FAN_BLOCK = 256;  // CSR entries (threads) per fan block

// vector types with explicit alignment (CUDA 13 deprecates the unsuffixed double4)
struct alignas(32) D4 {
  double x, y, z, w;
};

struct GatherPlan {
  int rows_per_block = 0;     // threads per block = rows per block
  int max_block_entries = 0;  // max over blocks of the CSR entries of the block's rows
  int max_block_steps = 0;    // max over blocks of the walk steps of the block's rows
  int w = 0;                  // slots per row of the layout (>= the longest row the kernels take, and
                              // large enough that every block's entries fit R * w)
  int64_t n_blocks = 0;
};

// diag_pos value of a row the row gather leaves out ("long row": more than
// 32 entries, or a star whose walk does not encode): the kernels give it no
// elements and zero its slice; long_rows_kernel computes it afterwards
constexpr uint8_t DIAG_LONG = 0xff;

// Shared-memory layout of one row-gather block: R rows (one per thread), W
// slots per row (the longest row of the mesh), L CSR entries and S walk
// steps.  Slot q of row t lives at index q * R + t ("thread-interleaved"), so
// the lanes of a warp touch consecutive records whichever slot each lane
// uses: the element loop is free of shared-memory bank conflicts.
//   nb0   T[4] per slot: edge vector d = x_j - x_i and u_x of the neighbour
//   nb1   T[2] per slot: u_y, u_z
//   acc   accumulators per slot (ab bytes): A and the three sums of c_i
//   col   int32 per CSR entry, read only while the records are gathered: it
//         shares nb1's bytes (nb1 is written after a barrier)
//   walk  one byte per step (copied as aligned 4-byte words, so S + 8 bytes)
//   stat  (time-step kernels only) the block's slice of A_static
// After the element loop, nb0 is reused to stage the finished values in CSR
// order for the coalesced write-out.
// Used identically by the host (launch size) and the kernel (carving).
struct GatherSmem {
  int R, W, L, S, tb, ab, ob, cr;  // ob: bytes of an output value; cr: components staged per write-out round
  int xs;                          // bytes per CSR entry of the time step's static slice (0: none)
  __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ size_t N() const { return (size_t)R * W; }
  __host__ __device__ size_t nb0() const { return 0; }
  __host__ __device__ size_t nb1() const { return up16(nb0() + (size_t)4 * tb * N()); }
  __host__ __device__ size_t acc() const { return up16(nb1() + (size_t)2 * tb * N()); }
  __host__ __device__ size_t col() const { return nb1(); }  // (L <= N: 4 L bytes fit in nb1)
  __host__ __device__ size_t walk() const { return up16(acc() + (size_t)ab * N()); }
  __host__ __device__ size_t stat() const { return up16(walk() + (size_t)S + 8); }
  __host__ __device__ size_t total() const { return up16(stat() + (size_t)xs * L); }
  // the write-out stages cr components of the block's L entries in nb0
  __host__ __device__ size_t stage_bytes() const { return (size_t)cr * L * ob; }
  __host__ __device__ bool stage_fits() const { return stage_bytes() <= nb1() - nb0(); }
};

// step: the layout of the time-step kernels (one accumulator per slot, at the
// 16-byte stride of the staged record halves; FP64 two planes of 16)
__host__ __device__ inline GatherSmem gather_smem(int precision, int R, int W, int L, int S, bool step = false) {
  GatherSmem g;
  g.R = R;
  g.W = W;
  g.L = L;
  g.S = S;
  g.tb = precision == NSI_FP64 ? 8 : 4;
  // accumulator bytes per slot: FP64 (A, G_x, G_y, G_z) doubles; the mixed
  // modes a float4 (G_x, G_y, G_z, A)
  g.ab = precision == NSI_FP64 ? 32 : 16;
  if (step) g.ab = precision == NSI_FP64 ? 32 : 16;
  g.xs = 0;
  g.ob = precision == NSI_MIXED_F32_ACC32 ? 4 : 8;
  g.cr = precision == NSI_MIXED_F32_ACC64 ? 2 : 4;
  if (step) g.xs = g.ob;  // the block's slice of A_static, copied in before the walk
  return g;
}

int gather_kernel_regs(int precision);  // registers per thread of the row-gather kernel

}  // namespace nsi

struct NsiHandle {
  int device = 0;
  int64_t n = 0, E = 0, nnz = 0;
  int precision = NSI_FP64;
  int scatter = NSI_SCATTER_AUTO;
  int block = 256;
  int debug = 0;
  int max_row = 0;
  int n_colors = 0;
  bool gather_ok = false;
  int64_t device_bytes = 0;

  // CSR pattern
  int32_t* row_ptr = nullptr;  // [n+1]
  int32_t* col_idx = nullptr;  // [nnz]
  // connectivity copy and colouring
  int4* lnods = nullptr;        // [E]
  int32_t* color_elems = nullptr;  // [E] element ids grouped by colour
  std::vector<int64_t> color_off;  // host [n_colors + 1]
  // row-gather map: every row's element walk (one byte per step)
  int32_t* walk_ptr = nullptr;  // [n+1]
  uint8_t* walk = nullptr;      // [walk_ptr[n] + 8]
  uint8_t* diag_pos = nullptr;  // [n] position of the diagonal inside its row (rows <= 32 entries)
  unsigned long long* elem_pos = nullptr;  // [E] element-position map (rows <= 32 entries), or null
  // edge-fan map (one word per CSR entry) and its block partition of the rows
  bool fan_ok = false;
  uint32_t* fan = nullptr;      // [nnz]
  int32_t* fan_blk = nullptr;   // [fan_blocks + 1] first row of every fan block
  int64_t fan_blocks = 0;
  bool use_fan = false;         // row-gather mode runs the edge-fan kernel
  bool atomic_agg = false;      // atomic mode runs the warp-aggregated atomics (else one atomic per value)
  bool persistent = false;      // row-gather mode runs the persistent grid (set by create: mixed64)
  int64_t long_rows = 0;        // rows the row gather leaves out, recomputed by long_rows_kernel
  int32_t* long_list = nullptr;  // [long_rows] their node ids
  int32_t* long_ptr = nullptr;   // [long_rows + 1] into long_inc
  uint32_t* long_inc = nullptr;  // element * 4 + local index of the row's node
  int64_t n_bad = 0;            // mixed modes: badly shaped elements (the adjoint and residual take them in double)
  int32_t* bad_list = nullptr;  // [n_bad] their ids
  uint32_t* bad_mask = nullptr; // [ceil(E / 32)] one bit per element, or null when there are none
  int64_t exact_rows = 0;       // mixed modes: rows recomputed in double (badly shaped elements)
  int32_t* exact_list = nullptr;  // [exact_rows] their node ids
  int32_t* exact_ptr = nullptr;   // [exact_rows + 1] into exact_inc
  uint32_t* exact_inc = nullptr;  // element * 4 + local index of the row's node
  // the stabilised block's row kernel: every row's star as row positions of
  // each element's other three nodes (five bits each, the row's node and the
  // three in a positively oriented order), and its warp tasks (one row, or two
  // consecutive rows of at most 16 entries), each described by two int4:
  // {first row, CSR start of the first row, of the second, end} and
  // {star start of the first row, of the second, end, diagonal positions |
  // rows << 16 | long << 24}
  uint16_t* star_word = nullptr;  // [incidences]
  int4* star_task = nullptr;      // [2 n_star_tasks]
  int64_t n_star_tasks = 0;
  nsi::GatherPlan plan;         // the launch plan in use
  nsi::GatherPlan plans[4];     // every rows-per-block candidate that fits shared memory
  int n_plans = 0;
  // coordinates: double4 for FP64, float4 hi + float4 lo for the mixed modes
  nsi::D4* xyz64 = nullptr;
  float4* xyz_hi = nullptr;
  float4* xyz_lo = nullptr;
  // per-call node records for the row-gather kernel (one 32-byte record per node
  // in the mixed modes, 64 bytes in FP64): coordinates and velocity of a node
  // in one or two DRAM sectors, rebuilt at the start of every gather call
  void* rec = nullptr;
  int rec_bytes = 0;
  // optional profiling events around the main assembly kernel
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
  // device error word
  unsigned* err = nullptr;
  // staging for nsi_assemble_host (allocated on first use)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // host-buffer calls: the CSR row starts on the host, and a stream and
  // events on which finished chunks of the outputs go to the host while the
  // next chunk is assembled
  std::vector<int32_t> row_ptr_host;  // [n+1]
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t chunk_ev[8] = {};
};

namespace nsi {

// --------------------------------------------------- element arithmetic ---
// For a positively oriented tet with edge vectors d1, d2, d3 leaving vertex 0,
// the cofactor vectors c_b = det(J) grad N_b are
//   c1 = d2 x d3,  c2 = d3 x d1,  c3 = d1 x d2,  c0 = -(c1 + c2 + c3),
// det J = d1 . c1 and |T| = det J / 6.  With them the Galerkin P1 terms are
//   convection  rho int N_a (u_h . grad N_b) = rho/120 (S + u_a) . c_b,
//               S = sum_c u_c  (exact P1 mass moments int N_a N_c = |T|(1+d_ac)/20,
//               which the 4-point Gauss rule integrates exactly)
//   viscous     mu |T| grad N_a . grad N_b  = mu / (6 det) c_a . c_b
//   lumped mass rho |T| / (4 dt)            = rho det / (24 dt)
//   pressure gradient  -int d_d N_a N_b     = -c_a[d] / 24  (every b)
//   lumped RHS  rho |T| u^n_a / (4 dt)      = rho det / (24 dt) u^n_a
template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__host__ __device__ __forceinline__ V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__host__ __device__ __forceinline__ T dot(const V3<T>& a, const V3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> add(const V3<T>& a, const V3<T>& b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}
template <typename T>
__host__ __device__ __forceinline__ V3<T> sub(const V3<T>& a, const V3<T>& b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}

// ------------------------------------------------ f32 -> f64 without DP ops ---
// GB300 executes double-precision instructions (including conversions) at a
// small fraction of the single-precision rate, so the mixed modes build their
// double outputs from integer operations on the IEEE-754 bit patterns.

// Exact float -> double (every float is a double).  Subnormal floats are
// renormalised; inf/nan keep their class.
__device__ __forceinline__ long long f32_to_f64_bits(float f) {
  unsigned u = __float_as_uint(f);
  unsigned sign = u & 0x80000000u;
  unsigned e = (u >> 23) & 0xffu;
  unsigned m = u & 0x7fffffu;
  unsigned e64;
  if (e == 0u) {
    if (m == 0u) return (long long)((unsigned long long)sign << 32);
    int lz = __clz(m) - 8;  // shift that brings the leading 1 to bit 23
    m = (m << lz) & 0x7fffffu;
    e64 = 897u - (unsigned)lz;  // 1 - 127 + 1023 - lz
  } else if (e == 0xffu) {
    e64 = 0x7ffu;
  } else {
    e64 = e + 896u;  // 1023 - 127
  }
  unsigned hi = sign | (e64 << 20) | (m >> 3);
  unsigned lo = m << 29;
  return (long long)(((unsigned long long)hi << 32) | lo);
}


// error-free sum: s + e == a + b exactly (Knuth's TwoSum, 6 float ops)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

}  // namespace nsi
