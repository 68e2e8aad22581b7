// Device kernels and the per-call entry points of libnsi_assemble.
//
//   elem_kernel     one element per thread (calculate_transients ...
//                   perform_assembly_in_global_system of Listing 1 fused),
//                   scatter by global atomics or, colour by colour, by plain
//                   read-add-write (deterministic)
//   gather_kernel   one CSR row per thread: the row's owner walks every
//                   element around its node (the element walk built at
//                   create), accumulates the row privately and the block
//                   writes its contiguous slice of A, G and rhs once,
//                   coalesced (no atomics, no zeroing, deterministic)
//   gather_persistent_kernel  the same as a persistent grid (a CTA's next
//                   block of rows starts its copies under the current
//                   block's write-out)
//   fan_kernel      one CSR entry per thread, walking the ring of elements
//                   around its edge (autotuning candidate)
//   batched_kernel  the row gather over many meshes in one persistent launch
//                   (their node records packed by one batched_pack_kernel)
//   step_kernel     one time step with cached geometry (A_static + C(u),
//                   rhs), or the paper's per-node outputs
//   step_persistent_kernel  the same as a persistent grid (mixed32)
//   vjp_kernel      adjoint of R(u, mu) = A(u) u - b, element per thread
//   residual_kernel R(u, mu) without the matrix (both with an exact
//                   companion for badly shaped elements in double)
//   exact_rows_kernel, long_rows_kernel  rows recomputed or computed per
//                   thread in double: the mixed modes' rows of badly shaped
//                   elements, and rows beyond the walk (more than 32 entries)
//   stab_star_kernel  the stabilised velocity block (3x3 per CSR entry): one
//                   warp per row or pair of rows, each element evaluated
//                   once per row, entry sums from shared memory
//   stab_rows_kernel  the stabilised block of listed rows, one thread per
//                   row in double
//   gather_values_kernel, add_values_kernel  pack / add the interface-row
//                   values of the element-partition exchange
//
// Formulas: see the element-arithmetic comment in nsi_internal.cuh.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "nsi_internal.cuh"

namespace nsi {

// ------------------------------------------------------------ views ------
struct MeshView {
  int64_t n, E, nnz;
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ col_idx;
  const int4* __restrict__ lnods;
  const int32_t* __restrict__ walk_ptr;
  const uint8_t* __restrict__ walk;
  const uint8_t* __restrict__ diag_pos;
  const D4* __restrict__ xyz64;
  const float4* __restrict__ xyz_hi;
  const float4* __restrict__ xyz_lo;
  const void* __restrict__ rec;
  const uint32_t* __restrict__ fan;
  const int32_t* __restrict__ fan_blk;
  unsigned* err;
};

// Physical constants of the element formulas, precomputed on the host in
// double (the float copies are rounded once): rho/120 (convection), mu/6
// (viscous) and rho/(24 dt) (lumped mass).
struct FieldView {
  const void* u[3];
  const void* un[3];
  double kc, kmu, kmass;
  float kcf, kmuf, kmassf;
};

template <typename T>
__device__ __forceinline__ T kc_of(const FieldView& f) {
  if constexpr (sizeof(T) == 8) return f.kc;
  else return f.kcf;
}
template <typename T>
__device__ __forceinline__ T kmu_of(const FieldView& f) {
  if constexpr (sizeof(T) == 8) return f.kmu;
  else return f.kmuf;
}
template <typename T>
__device__ __forceinline__ T kmass_of(const FieldView& f) {
  if constexpr (sizeof(T) == 8) return f.kmass;
  else return f.kmassf;
}

struct OutView {
  void* A;
  void* G;
  void* rhs;
};

static MeshView view_of(const NsiHandle* h) {
  MeshView m;
  m.n = h->n;
  m.E = h->E;
  m.nnz = h->nnz;
  m.row_ptr = h->row_ptr;
  m.col_idx = h->col_idx;
  m.lnods = h->lnods;
  m.walk_ptr = h->walk_ptr;
  m.walk = h->walk;
  m.diag_pos = h->diag_pos;
  m.xyz64 = h->xyz64;
  m.xyz_hi = h->xyz_hi;
  m.xyz_lo = h->xyz_lo;
  m.rec = h->rec;
  m.fan = h->fan;
  m.fan_blk = h->fan_blk;
  m.err = h->err;
  return m;
}

static FieldView fields_of(const NsiFields* f) {
  FieldView v;
  for (int k = 0; k < 3; ++k) {
    v.u[k] = f->u[k];
    v.un[k] = f->u_n[k] ? f->u_n[k] : f->u[k];
  }
  v.kc = f->rho / 120.0;
  v.kmu = f->mu / 6.0;
  v.kmass = f->rho / (24.0 * f->dt);
  v.kcf = (float)v.kc;
  v.kmuf = (float)v.kmu;
  v.kmassf = (float)v.kmass;
  return v;
}

// precision traits: compute type T, output type Out
template <int P>
struct Prec;
template <>
struct Prec<NSI_FP64> {
  using T = double;
  using Out = double;
};
template <>
struct Prec<NSI_MIXED_F32_ACC64> {
  using T = float;
  using Out = double;
};
template <>
struct Prec<NSI_MIXED_F32_ACC32> {
  using T = float;
  using Out = float;
};

template <typename T>
__device__ __forceinline__ T rcp(T x);
template <>
__device__ __forceinline__ float rcp<float>(float x) {
  return __frcp_rn(x);
}
template <>
__device__ __forceinline__ double rcp<double>(double x) {
  return 1.0 / x;
}

// node coordinates: exact double, or a float hi/lo pair whose difference
// gives edge vectors to ~2^-48 relative before the float arithmetic starts
template <int P>
struct NodeX;
template <>
struct NodeX<NSI_FP64> {
  V3<double> x;
  __device__ __forceinline__ void load(const MeshView& m, int64_t v) {
    D4 p = m.xyz64[v];
    x = {p.x, p.y, p.z};
  }
  __device__ __forceinline__ V3<double> minus(const NodeX& o) const { return sub(x, o.x); }
};
template <int P>
struct NodeX {
  V3<float> hi, lo;
  __device__ __forceinline__ void load(const MeshView& m, int64_t v) {
    float4 a = __ldg(m.xyz_hi + v);
    float4 b = __ldg(m.xyz_lo + v);
    hi = {a.x, a.y, a.z};
    lo = {b.x, b.y, b.z};
  }
  __device__ __forceinline__ V3<float> minus(const NodeX& o) const { return add(sub(hi, o.hi), sub(lo, o.lo)); }
};

template <typename T>
__device__ __forceinline__ V3<T> load_vec(const void* const* comp, int64_t v) {
  return {__ldg(static_cast<const T*>(comp[0]) + v), __ldg(static_cast<const T*>(comp[1]) + v),
          __ldg(static_cast<const T*>(comp[2]) + v)};
}

// asynchronous global -> shared copies (cp.async): many gathers in flight per
// thread without holding registers
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most the most recent committed group is still in flight
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---------------------------------------------------------- node records ---
// One record per node, rebuilt every call from the handle's coordinates and
// the caller's velocities, so that the row-gather kernel fetches a neighbour
// with one 32-byte (mixed) or 64-byte (FP64) request instead of five:
//   mixed: {hx, hy, hz, ux} {uy, uz, lo_xy, lo_z}, lo_* the top 16 bits of
//          the float low parts (coordinates kept to ~2^-32 relative)
//   FP64:  {x, y, z, 0} {ux, uy, uz, 0} as doubles
template <int P>
__device__ __forceinline__ void pack_node(const MeshView& m, const FieldView& f, void* __restrict__ rec, int64_t i) {
  if constexpr (P == NSI_FP64) {
    const D4 x = m.xyz64[i];
    const V3<double> u = load_vec<double>(f.u, i);
    D4* r = static_cast<D4*>(rec) + 2 * i;
    r[0] = D4{x.x, x.y, x.z, 0.0};
    r[1] = D4{u.x, u.y, u.z, 0.0};
  } else {
    const float4 hi = __ldg(m.xyz_hi + i);
    const float4 lo = __ldg(m.xyz_lo + i);
    const V3<float> u = load_vec<float>(f.u, i);
    uint4* r = static_cast<uint4*>(rec) + 2 * i;
    r[0] = make_uint4(__float_as_uint(hi.x), __float_as_uint(hi.y), __float_as_uint(hi.z), __float_as_uint(u.x));
    r[1] = make_uint4(__float_as_uint(u.y), __float_as_uint(u.z),
                      (__float_as_uint(lo.x) >> 16) | (__float_as_uint(lo.y) & 0xffff0000u),
                      __float_as_uint(lo.z) & 0xffff0000u);
  }
}

template <int P>
__global__ void __launch_bounds__(256) pack_kernel(MeshView m, FieldView f, void* __restrict__ rec) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m.n) pack_node<P>(m, f, rec, i);
}

__device__ __forceinline__ V3<float> record_lo(float w6, float w7) {
  const unsigned a = __float_as_uint(w6), b = __float_as_uint(w7);
  return {__uint_as_float(a << 16), __uint_as_float(a & 0xffff0000u), __uint_as_float(b & 0xffff0000u)};
}

// ------------------------------------------------ element-centric kernel ---
template <typename T, typename Out>
__device__ __forceinline__ void add_out(Out* p, T v, bool atomic);

template <>
__device__ __forceinline__ void add_out<double, double>(double* p, double v, bool atomic) {
  if (atomic) atomicAdd(p, v);
  else *p += v;
}
template <>
__device__ __forceinline__ void add_out<float, float>(float* p, float v, bool atomic) {
  if (atomic) atomicAdd(p, v);
  else *p += v;
}
// an element value in the output type (float -> double exactly)
template <typename T, typename Out>
__device__ __forceinline__ Out to_out(T v) {
  if constexpr (sizeof(T) == sizeof(Out)) return v;
  else return __longlong_as_double(f32_to_f64_bits(v));
}
template <>
__device__ __forceinline__ void add_out<float, double>(double* p, float v, bool atomic) {
  double d = __longlong_as_double(f32_to_f64_bits(v));
  if (atomic) atomicAdd(p, d);  // the add itself happens in the L2 atomic unit
  else *p += d;
}

// Warp-aggregated global add: the lanes of a warp whose `key` (the output
// position) is equal form a group (__match_any_sync); the group's lowest lane
// collects the others' values by shuffles, in lane order, and issues one
// atomic add per value, value k to dst[k] (the same address in every lane of
// a group: it is a function of the key).  Every lane of the warp takes part
// (a lane with nothing to add passes a key of its own and valid = false).
template <int V, typename Out>
__device__ __forceinline__ void warp_aggregated_add(Out* const (&dst)[V], int64_t key, const Out (&val)[V],
                                                    bool valid) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  Out sum[V];
#pragma unroll
  for (int k = 0; k < V; ++k) sum[k] = val[k];
  unsigned others = peers & (peers - 1u);  // the group's lanes after its leader
  while (__any_sync(0xffffffffu, others != 0u)) {
    const int src = others ? __ffs(others) - 1 : (int)lane;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const Out v = __shfl_sync(0xffffffffu, val[k], src);
      if (others) sum[k] += v;
    }
    others &= others - 1u;
  }
  if (valid && lane == (unsigned)(__ffs(peers) - 1)) {
#pragma unroll
    for (int k = 0; k < V; ++k) atomicAdd(dst[k], sum[k]);
  }
}

// One element per thread (the Listing 1 subroutines fused).  Each of the 16
// (row, column) entries of the element is located in the CSR pattern through
// the element-position map (or, for rows longer than 32 entries, a scan of
// the row), and its A value and three G values are added:
//   ATOMIC: by global atomic adds, one per value, or with AGG by
//           warp-aggregated atomics (the elements of a warp are consecutive
//           in the mesh's order, so neighbouring elements share entries;
//           every group of lanes adding to one entry issues one atomic per
//           value) -- the scatter's order is not deterministic;
//   otherwise (one colour of a colouring: no two elements of the launch share
//           a node) by plain read-add-write, deterministic.
// In mixed64 the float element values are converted to double exactly
// before they are summed (the accumulation is in double).
template <int P, bool ATOMIC, bool DEBUG, bool AGG = false>
__global__ void __launch_bounds__(256) elem_kernel(MeshView m, FieldView f, OutView o,
                                                   const int32_t* __restrict__ elems, int64_t count,
                                                   const unsigned long long* __restrict__ elem_pos) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool valid = t < count;
  if (!ATOMIC && !valid) return;  // (the atomic path keeps whole warps for the aggregation)
  const int64_t e = valid ? (elems ? (int64_t)elems[t] : t) : 0;
  const int4 q = valid ? m.lnods[e] : make_int4(0, 0, 0, 0);
  const int v[4] = {q.x, q.y, q.z, q.w};
  if (DEBUG && valid) {
    for (int a = 0; a < 4; ++a)
      if (v[a] < 0 || v[a] >= m.n) {
        atomicOr(m.err, ERR_BAD_INDEX);
        valid = false;
      }
    if (!valid) {
      if (!ATOMIC) return;
    }
  }
  const int vv[4] = {valid ? v[0] : 0, valid ? v[1] : 0, valid ? v[2] : 0, valid ? v[3] : 0};
  // gather (calculate_transients)
  NodeX<P> X[4];
  V3<T> u[4], un[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a].load(m, vv[a]);
    u[a] = load_vec<T>(f.u, vv[a]);
    un[a] = load_vec<T>(f.un, vv[a]);
  }
  // Jacobian columns, cofactors, det (calculate_cartesian_derivatives)
  const V3<T> d1 = X[1].minus(X[0]), d2 = X[2].minus(X[0]), d3 = X[3].minus(X[0]);
  V3<T> c[4];
  c[1] = cross(d2, d3);
  c[2] = cross(d3, d1);
  c[3] = cross(d1, d2);
  const T det = dot(d1, c[1]);
  c[0] = {-(c[1].x + c[2].x + c[3].x), -(c[1].y + c[2].y + c[3].y), -(c[1].z + c[2].z + c[3].z)};
  // Gauss-point velocity moments and element matrices
  const V3<T> S = add(add(u[0], u[1]), add(u[2], u[3]));
  const T kc = kc_of<T>(f);
  const T kv = kmu_of<T>(f) * rcp(valid ? det : T(1));
  const T km = det * kmass_of<T>(f);
  const T kg = (T)(-1.0 / 24.0);
  Out* A = static_cast<Out*>(o.A);
  Out* G = static_cast<Out*>(o.G);
  Out* R = static_cast<Out*>(o.rhs);
  // perform_assembly_in_global_system: the 16 positions of the element's entries
  int pos[4][4];
  if (elem_pos) {
    const unsigned long long w = valid ? elem_pos[e] : 0ull;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int rs = m.row_ptr[vv[a]];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        pos[a][b] = rs + (b == a ? (int)m.diag_pos[vv[a]]
                                 : (int)((w >> (ELEM_POS_BITS * elem_pos_slot(a, b))) & 31ull));
    }
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = vv[a];
      const int rs = m.row_ptr[r], re = m.row_ptr[r + 1];
#pragma unroll
      for (int b = 0; b < 4; ++b) pos[a][b] = -1;
      for (int s2 = rs; s2 < re; ++s2) {
        const int cidx = m.col_idx[s2];
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (cidx == vv[b]) pos[a][b] = s2;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const V3<T> va = add(S, u[a]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      bool ok = valid;
      if (DEBUG && ok && pos[a][b] < 0) {
        atomicOr(m.err, ERR_NOT_IN_PATTERN);
        ok = false;
      }
      T Aab = kc * dot(va, c[b]) + kv * dot(c[a], c[b]);
      if (a == b) Aab += km;
      const T g3[3] = {kg * c[a].x, kg * c[a].y, kg * c[a].z};
      if constexpr (ATOMIC) {
        Out vals[4];
        vals[0] = to_out<T, Out>(Aab);
#pragma unroll
        for (int d = 0; d < 3; ++d) vals[d + 1] = to_out<T, Out>(g3[d]);
        const int64_t key = ok ? (int64_t)pos[a][b] : -1 - (int64_t)(threadIdx.x & 31u);
        const int64_t pk = ok ? key : 0;
        Out* const dst[4] = {A + pk, G + pk, G + m.nnz + pk, G + 2 * m.nnz + pk};
        if constexpr (AGG) {
          warp_aggregated_add<4, Out>(dst, key, vals, ok);
        } else if (ok) {
#pragma unroll
          for (int k = 0; k < 4; ++k) atomicAdd(dst[k], vals[k]);
        }
      } else if (ok) {
        add_out<T, Out>(A + pos[a][b], Aab, false);
#pragma unroll
        for (int d = 0; d < 3; ++d) add_out<T, Out>(G + d * m.nnz + pos[a][b], g3[d], false);
      }
    }
    const T r3[3] = {km * un[a].x, km * un[a].y, km * un[a].z};
    if constexpr (ATOMIC) {
      Out rv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) rv[k] = to_out<T, Out>(r3[k]);
      const int64_t key = valid ? (int64_t)vv[a] : -1 - (int64_t)(threadIdx.x & 31u);
      Out* const dst[3] = {R + vv[a], R + m.n + vv[a], R + 2 * m.n + vv[a]};
      if constexpr (AGG) {
        warp_aggregated_add<3, Out>(dst, key, rv, valid);
      } else if (valid) {
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(dst[k], rv[k]);
      }
    } else if (valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k) add_out<T, Out>(R + k * m.n + vv[a], r3[k], false);
    }
  }
}

// ---------------------------------------------------- row-gather kernel ---
// Register accumulator of one output value: plain T, or a compensated float
// pair (TwoSum) for the mixed mode with double output.
template <int P>
struct Acc {
  using T = typename Prec<P>::T;
  T v;
  __device__ __forceinline__ void zero() { v = T(0); }
  __device__ __forceinline__ void add(T x) { v += x; }
};
template <>
struct Acc<NSI_MIXED_F32_ACC64> {
  float hi, lo;
  __device__ __forceinline__ void zero() { hi = lo = 0.0f; }
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
};

__device__ __forceinline__ void store_acc(double* p, const Acc<NSI_FP64>& a) { *p = a.v; }
__device__ __forceinline__ void store_acc(float* p, const Acc<NSI_MIXED_F32_ACC32>& a) { *p = a.v; }
// The double nearest hi + lo for a renormalised float pair (|lo| <= ulp(hi) /
// 2) with a finite hi, without branches: the double of |hi| from its bits, lo
// (with hi's sign taken out) added as an integer k of the double's units in
// the last place (|k| <= 2^28), hi's sign set last.  When |hi| is a power of
// two and the sum lies below it, k counts the half-size units of the binade
// below.  Zero gives zero; a tiny |hi| (below 2^-75, where the scale of k would
// leave the float range) is handled at 2^100 times its size, the exponent
// taken back in the result.  Infinite and NaN values are the callers' (a test
// for them here costs the write-out loop several percent).
__device__ __forceinline__ double normalised_pair_double(float hi, float lo) {
  const unsigned u0 = __float_as_uint(hi);
  const bool tiny = ((u0 >> 23) & 0xffu) < 52u;
  const float sc = tiny ? 0x1p100f : 1.0f;
  const float h2 = hi * sc, l2 = lo * sc;  // exact
  const unsigned uh = __float_as_uint(h2);
  const unsigned eh = (uh >> 23) & 0xffu;
  const float ls = __uint_as_float(__float_as_uint(l2) ^ (uh & 0x80000000u));
  const unsigned below = ((uh << 9) == 0u && ls < 0.0f) ? 1u : 0u;
  const int k = __float2int_rn(ls * __uint_as_float((306u + below - eh) << 23));
  const unsigned long long mag =
      ((unsigned long long)(uh & 0x7fffffffu) << 29) + ((tiny ? 796ull : 896ull) << 52);
  const unsigned long long r = (mag + (unsigned long long)(long long)k) | ((unsigned long long)(uh & 0x80000000u) << 32);
  return __longlong_as_double((u0 << 1) == 0u ? (long long)((unsigned long long)(u0 & 0x80000000u) << 32)
                                              : (long long)r);
}
// an infinite or NaN accumulator (hi) as a double of the same class
__device__ __forceinline__ double nonfinite_double(float hi) { return __longlong_as_double(f32_to_f64_bits(hi)); }
// true if the exponent bits of x are all ones (infinite or NaN)
__device__ __forceinline__ bool nonfinite_bits(float x) { return (__float_as_uint(x) | 0x807fffffu) == 0xffffffffu; }
// true for an infinite, NaN or subnormal float (the cases float_double leaves out)
__device__ __forceinline__ bool special_float(float x) {
  const unsigned e = __float_as_uint(x) & 0x7f800000u;
  return e == 0x7f800000u || (e == 0u && (__float_as_uint(x) & 0x007fffffu) != 0u);
}
// the double equal to a normal or zero float, from its bit pattern: the
// exponent rebiased (+896), the 23 mantissa bits moved to the top of the
// double's 52; the sign kept.  A subnormal float (below 2^-126 in magnitude)
// gives a signed zero; infinite and NaN floats are not handled (the values
// converted this way are the pressure-gradient sums, functions of the
// coordinates a handle validates, far inside the float range for any mesh
// whose float element arithmetic is meaningful).
__device__ __forceinline__ double float_double(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned a = u & 0x7fffffffu;
  const unsigned hi = (a < 0x00800000u ? 0u : (a >> 3) + (896u << 20)) | (u & 0x80000000u);
  return __hiloint2double((int)hi, a < 0x00800000u ? 0 : (int)(u << 29));
}
// the double nearest hi + lo of a pair with a finite hi: renormalised first
// (Fast2Sum)
__device__ __forceinline__ double pair_double(float hi, float lo) {
  const float s = hi + lo;
  const float l = lo - (s - hi);
  return normalised_pair_double(s, l);
}
__device__ __forceinline__ void store_acc(double* p, const Acc<NSI_MIXED_F32_ACC64>& a) {
  *p = nonfinite_bits(a.hi) ? nonfinite_double(a.hi) : pair_double(a.hi, a.lo);
}

template <typename T>
struct alignas(4 * sizeof(T)) T4 {
  T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) T2 {
  T x, y;
};

// Accumulators of the block's slots in shared memory: the A value and the
// pressure-gradient values (sums of -c_i / 24) of each entry.  A slot is only
// touched by the thread owning its row until the final write-out, so no
// atomics are needed.  add3() updates three DISTINCT slots (the three other
// nodes of one element sit at three different positions of the row), so all
// three loads are issued before the stores.
template <int P>
struct AccSmem;
// paired float arithmetic (one instruction for two lanes of a float2, each
// rounded like its scalar counterpart); a - b is formed as b * (-1) + a with a
// single rounding
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// error-free sum of pairs (TwoSum lane by lane): h + x = s + e exactly; s
// replaces h and e is added to the error term l
__device__ __forceinline__ void two_sum2(float2& h, float2& l, float2 x) {
  const float2 s = add2(h, x);
  const float2 bb = sub2(s, h);
  const float2 e = add2(sub2(h, sub2(s, bb)), sub2(x, bb));
  h = s;
  l = add2(l, e);
}

// Float slots hold (G_x, G_y, G_z, A): the two halves are
// the pairs (G_x, G_y) and (G_z, A) of the paired updates.
template <>
struct AccSmem<NSI_MIXED_F32_ACC32> {
  float4* __restrict__ a;
  __device__ __forceinline__ AccSmem(unsigned char* p, size_t) : a(reinterpret_cast<float4*>(p)) {}
  __device__ __forceinline__ void zero(int k) { a[k] = make_float4(0.f, 0.f, 0.f, 0.f); }
  struct Slot {
    float2 g, r;  // (G_x, G_y), (G_z, A)
  };
  __device__ __forceinline__ Slot load1(int k) const {
    const float4 v = a[k];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
  }
  __device__ __forceinline__ void store1(int k, const Slot& v) { a[k] = make_float4(v.g.x, v.g.y, v.r.x, v.r.y); }
  static __device__ __forceinline__ void add(Slot& s, float2 gxy, float2 gz_a) {
    s.g = add2(s.g, gxy);
    s.r = add2(s.r, gz_a);
  }
  // sums over the row's slots t, t + R, ... (len of them), the diagonal's
  // included: it is still zero here (zeroed with the others; the walk only
  // ever adds zeros to it), so no test is needed (r[0]: A, r[1..3]: G_x..G_z)
  __device__ __forceinline__ void row_sums(int t, int R, int len, Acc<NSI_MIXED_F32_ACC32>* r) const {
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) {
      const float4 v = a[k];
      r[0].add(v.w); r[1].add(v.x); r[2].add(v.y); r[3].add(v.z);
    }
  }
  __device__ __forceinline__ void set(int k, const Acc<NSI_MIXED_F32_ACC32>* r) {
    a[k] = make_float4(r[1].v, r[2].v, r[3].v, r[0].v);
  }
  // finished values (A, G_x, G_y, G_z) of slot k
  __device__ __forceinline__ T4<float> values(int k) const {
    const float4 v = a[k];
    return {v.w, v.x, v.y, v.z};
  }
};
// mixed64: float slots (G_x, G_y, G_z, A) as mixed32.  An off-diagonal entry
// sums the ~5 element terms of its edge (float products), so its float sum
// carries a few roundings of those terms; the cancellation is in the
// diagonal, the lumped mass minus the row's other entries, which row_sums
// forms as a compensated sum (TwoSum over the row's entries, about 48
// significant bits).  The diagonal's error term stays in a register of the
// row's thread (dlo) until the write-out converts the pair to double.
template <>
struct AccSmem<NSI_MIXED_F32_ACC64> {
  float4* __restrict__ hi;  // (G_x, G_y, G_z, A)
  float dlo = 0.f;          // error term of this thread's diagonal A (set())
  __device__ __forceinline__ AccSmem(unsigned char* p, size_t) : hi(reinterpret_cast<float4*>(p)) {}
  __device__ __forceinline__ void zero(int k) { hi[k] = make_float4(0.f, 0.f, 0.f, 0.f); }
  struct Slot {
    float2 g, r;  // (G_x, G_y), (G_z, A)
  };
  __device__ __forceinline__ Slot load1(int k) const {
    const float4 h = hi[k];
    return {make_float2(h.x, h.y), make_float2(h.z, h.w)};
  }
  __device__ __forceinline__ void store1(int k, const Slot& v) { hi[k] = make_float4(v.g.x, v.g.y, v.r.x, v.r.y); }
  static __device__ __forceinline__ void add(Slot& s, float2 gxy, float2 gz_a) {
    s.g = add2(s.g, gxy);
    s.r = add2(s.r, gz_a);
  }
  // sums over the row's slots, the diagonal's included (still zero): A
  // compensated, G plain (r[0]: A, r[1..3]: G_x..G_z with zero error terms)
  __device__ __forceinline__ void row_sums(int t, int R, int len, Acc<NSI_MIXED_F32_ACC64>* r) const {
    float2 g = make_float2(0.f, 0.f), za = g;
    float al = 0.f;
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) {
      const float4 h = hi[k];
      g = add2(g, make_float2(h.x, h.y));
      const float2 t2 = add2(za, make_float2(h.z, h.w));
      const float bb = t2.y - za.y;
      al += (za.y - (t2.y - bb)) + (h.w - bb);
      za = t2;
    }
    r[0].hi = za.y; r[0].lo = al;
    r[1].hi = g.x; r[1].lo = 0.f;
    r[2].hi = g.y; r[2].lo = 0.f;
    r[3].hi = za.x; r[3].lo = 0.f;
  }
  // the diagonal: A's leading part and G in the slot, A's error term kept
  __device__ __forceinline__ void set(int k, const Acc<NSI_MIXED_F32_ACC64>* r) {
    hi[k] = make_float4(r[1].hi, r[2].hi, r[3].hi, r[0].hi);
    dlo = r[0].lo;
  }
};
template <>
struct AccSmem<NSI_FP64> {
  T2<double>* __restrict__ a0;  // A, G_x
  T2<double>* __restrict__ a1;  // G_y, G_z
  __device__ __forceinline__ AccSmem(unsigned char* p, size_t N)
      : a0(reinterpret_cast<T2<double>*>(p)), a1(reinterpret_cast<T2<double>*>(p) + N) {}
  __device__ __forceinline__ void zero(int k) {
    a0[k] = {0.0, 0.0};
    a1[k] = {0.0, 0.0};
  }
  struct Slot {
    T2<double> x, y;  // (A, G_x), (G_y, G_z)
  };
  __device__ __forceinline__ Slot load1(int k) const { return {a0[k], a1[k]}; }
  __device__ __forceinline__ void store1(int k, const Slot& v) {
    a0[k] = v.x;
    a1[k] = v.y;
  }
  static __device__ __forceinline__ void update1(Slot& s, double A, double gx, double gy, double gz) {
    s.x.x += A; s.x.y += gx; s.y.x += gy; s.y.y += gz;
  }
  __device__ __forceinline__ void row_sums(int t, int R, int len, Acc<NSI_FP64>* r) const {
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) {
      const T2<double> x = a0[k], y = a1[k];
      r[0].add(x.x); r[1].add(x.y); r[2].add(y.x); r[3].add(y.y);
    }
  }
  __device__ __forceinline__ void set(int k, const Acc<NSI_FP64>* r) {
    a0[k] = {r[0].v, r[1].v};
    a1[k] = {r[2].v, r[3].v};
  }
  __device__ __forceinline__ T4<double> values(int k) const {
    const T2<double> x = a0[k], y = a1[k];
    return {x.x, x.y, y.x, y.y};
  }
};

// where the second half of a neighbour's record lands before the edge vectors
// are formed: inside the slot's accumulators, which are zeroed right after
template <int P>
__device__ __forceinline__ void* staged_half(unsigned char* smem, const GatherSmem& lay, int k, int part) {
  if constexpr (P == NSI_FP64) return reinterpret_cast<T2<double>*>(smem + lay.acc()) + (size_t)part * lay.N() + k;
  else return reinterpret_cast<float4*>(smem + lay.acc()) + k;
}

// reciprocal of det: the float path uses the fast approximate division
// (about 1 ulp); the double path refines the hardware's approximate double
// reciprocal (rcp.approx.ftz.f64, relative error at most 2^-20 over 4 M
// normal inputs measured on GB300) by two Newton-Raphson steps for 1/x,
// r <- r + r (1 - x r), each of which squares the relative error (2^-40,
// then below the double's rounding): four FMAs instead of the IEEE
// division's longer sequence on GB300's slow FP64 pipe (3.18 -> 3.15 ms at
// the 100^3 cube).  det is a normal number here (the mesh is validated at
// create).
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_fast(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
#pragma unroll
  for (int it = 0; it < 2; ++it) r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// The element walk of one row (the element loop of phase 2), node i as the
// origin.  A window of two neighbours (p, q) stays in registers with their
// edge vectors, velocities and accumulators; every step brings one node c in
// from shared memory, evaluates the element (i, p, q, c) if the step says so,
// then writes back the accumulator of the node that leaves the window; c
// always becomes q, and p keeps its node or takes q's (one register move of
// a node per step instead of two selects).  With
// c_p = d_q x d_c, c_q = d_c x d_p, c_c = d_p x d_q (cofactors of the
// Jacobian, calculate_cartesian_derivatives, for the order (p, q, c)),
// det = d_p . c_p and c_i = -(c_p + c_q + c_c), the element adds
//   A(i,x) += w . c_x  (x = p, q, c),  w = rho/120 (2 u_i + u_p + u_q + u_c) + mu/(6 det) c_i
// (FP64: the staged velocities already carry the factor rho/120)
// -c_i / 24 (= -|T| grad N_i / 4, the element's G(i, x)) to the three
// pressure-gradient values and det to the lumped mass sum (scaled after the
// walk).  For the order (p, q, c) an odd permutation of the
// element's own, det and every cofactor change sign, w does not, so every
// contribution is multiplied by -1.  c_c is carried from the previous step:
// after q leaves, the window (p, c) has d_p x d_c = -c_q; after p leaves,
// (q, c) has d_q x d_c = c_p; m holds c_q or c_p and c_c = -sg m with sg = 1
// or -1.
template <typename T, typename Slot>
struct WalkNode {
  int k;  // shared-memory slot
  V3<T> d, u;
  Slot v;
};

template <int P>
__device__ __forceinline__ WalkNode<typename Prec<P>::T, typename AccSmem<P>::Slot> walk_load(
    int k, const T4<typename Prec<P>::T>* __restrict__ nb0, const T2<typename Prec<P>::T>* __restrict__ nb1,
    const AccSmem<P>& acc) {
  using T = typename Prec<P>::T;
  const T4<T> a = nb0[k];
  const T2<T> b = nb1[k];
  return {k, {a.x, a.y, a.z}, {a.w, b.x, b.y}, acc.load1(k)};
}

template <int P, bool DEBUG>
__device__ __forceinline__ void walk_row(const uint8_t* __restrict__ st, int nsteps, int len,
                                         const T4<typename Prec<P>::T>* __restrict__ nb0,
                                         const T2<typename Prec<P>::T>* __restrict__ nb1, AccSmem<P>& acc, int t,
                                         int R, const V3<typename Prec<P>::T>& u2i, typename Prec<P>::T kc,
                                         typename Prec<P>::T kmu, Acc<P>& detsum, unsigned* err) {
  using T = typename Prec<P>::T;
  using Node = WalkNode<T, typename AccSmem<P>::Slot>;
  constexpr T kg = T(-1.0 / 24.0);  // the pressure-gradient sums are accumulated scaled
  if (nsteps <= 0) return;
  if (DEBUG) {
    bool ok = nsteps >= 3 && !(st[0] & WALK_ELEM) && !(st[1] & WALK_ELEM);
    for (int s = 0; s < nsteps; ++s) ok &= (int)(st[s] & WALK_POS) < len;
    if (!ok) {
      atomicOr(err, ERR_STAR);
      return;
    }
  }
  if (nsteps < 3) return;  // (every walk of a row with elements has at least 3 steps)
  // a row's walk starts with two steps that only fill the window (the
  // encoder begins the first path that way): their nodes are loaded directly,
  // with the cofactor the first element carries, c_c = d_p x d_q
  Node p = walk_load<P>((int)(st[0] & WALK_POS) * R + t, nb0, nb1, acc);
  Node n0 = walk_load<P>((int)(st[1] & WALK_POS) * R + t, nb0, nb1, acc);
  V3<T> m = cross(p.d, n0.d);
  T sg = T(-1);  // c_c = -sg m
  unsigned w = st[2];
  Node n1 = walk_load<P>((int)(w & WALK_POS) * R + t, nb0, nb1, acc);
  Node n2;
  // One step: the element (i, p, q, c); the next step's node is loaded into
  // nx (in flight while the element is evaluated; never one of p, q, c: the
  // walk is encoded that way; the last step reloads its own node, unused).
  // Afterwards the window is (p, c): p keeps its node or takes q's.
  auto step = [&](Node& q, Node& c, Node& nx, int s) {
    const unsigned wn = st[s + 1 < nsteps ? s + 1 : s];
    nx = walk_load<P>((int)(wn & WALK_POS) * R + t, nb0, nb1, acc);
    const V3<T> cp = cross(q.d, c.d), cq = cross(c.d, p.d);
    const bool elem = (w & WALK_ELEM) != 0u;
    if constexpr (P == NSI_FP64) {
      if (elem) {  // (steps that only fill the window come first in a row: warp-uniform)
        const T det = dot(p.d, cp);
        const V3<T> ci{fma(sg, m.x, -(cp.x + cq.x)), fma(sg, m.y, -(cp.y + cq.y)), fma(sg, m.z, -(cp.z + cq.z))};
        const T kv = kmu * rcp_fast(det);
        const V3<T> w3{(u2i.x + p.u.x + q.u.x + c.u.x) + kv * ci.x, (u2i.y + p.u.y + q.u.y + c.u.y) + kv * ci.y,
                       (u2i.z + p.u.z + q.u.z + c.u.z) + kv * ci.z};
        const bool neg = (w & WALK_NEG) != 0u;  // orientation
        const T f = neg ? T(-1) : T(1), fg = neg ? -kg : kg;
        const T gx = fg * ci.x, gy = fg * ci.y, gz = fg * ci.z;
        AccSmem<P>::update1(p.v, f * dot(w3, cp), gx, gy, gz);
        AccSmem<P>::update1(q.v, f * dot(w3, cq), gx, gy, gz);
        AccSmem<P>::update1(c.v, -f * sg * dot(w3, m), gx, gy, gz);
        detsum.add(f * det);
      }
    } else {
      // branch-free: a step that only fills the window adds zeros
      const float det = dot(p.d, cp);
      const V3<float> ci{fmaf(sg, m.x, -(cp.x + cq.x)), fmaf(sg, m.y, -(cp.y + cq.y)), fmaf(sg, m.z, -(cp.z + cq.z))};
      const float kv = kmu * rcp_fast(elem ? det : 1.0f);
      const V3<float> w3{kc * (u2i.x + p.u.x + q.u.x + c.u.x) + kv * ci.x,
                         kc * (u2i.y + p.u.y + q.u.y + c.u.y) + kv * ci.y,
                         kc * (u2i.z + p.u.z + q.u.z + c.u.z) + kv * ci.z};
      const bool neg = (w & WALK_NEG) != 0u;
      const float f = elem ? (neg ? -1.0f : 1.0f) : 0.0f;  // orientation, or 0
      const float fg = elem ? (neg ? -kg : kg) : 0.0f;
      const float2 gg = make_float2(fg, fg), ff = make_float2(fg, f);
      const float2 gxy = __fmul2_rn(make_float2(ci.x, ci.y), gg);
      AccSmem<P>::add(p.v, gxy, __fmul2_rn(make_float2(ci.z, dot(w3, cp)), ff));
      AccSmem<P>::add(q.v, gxy, __fmul2_rn(make_float2(ci.z, dot(w3, cq)), ff));
      AccSmem<P>::add(c.v, gxy, __fmul2_rn(make_float2(ci.z, dot(w3, m)), make_float2(fg, -f * sg)));
      detsum.add(f * det);
    }
    const bool evq = (w & WALK_EVQ) != 0u;
    const Node& lv = evq ? q : p;  // the node that leaves the window
    acc.store1(lv.k, lv.v);
    if (!evq) p = q;
    m = evq ? cq : cp;
    sg = evq ? T(1) : T(-1);
    w = wn;
  };
  // The nodes q, c and the one in flight rotate through n0, n1, n2: three
  // steps per iteration bring them back to their places, so the newest node
  // never moves between registers (only p's update depends on the walk).
  int s = 2;
  for (; s + 3 <= nsteps; s += 3) {
    step(n0, n1, n2, s);
    step(n1, n2, n0, s + 1);
    step(n2, n0, n1, s + 2);
  }
  if (s < nsteps) {
    step(n0, n1, n2, s);
    if (s + 1 < nsteps) {
      step(n1, n2, n0, s + 1);
      acc.store1(n2.k, n2.v);
    } else {
      acc.store1(n1.k, n1.v);
    }
  } else {
    acc.store1(n0.k, n0.v);
  }
  acc.store1(p.k, p.v);
}

// Per-thread view of one block of rows [r0, r0 + blockDim.x) of one mesh.
template <typename T>
struct BlockRows {
  int R, t, nrows, L, len, lb, s0, s1, dp;
  int64_t i;
  int32_t base;
  V3<T> uni;
  int zl;  // a long row's entries (its slice is zeroed in the write-out; 0 for the others)
};

// Phase 0 of a block: its bounds and the row's scalars (plain loads, in
// flight until first used), then the asynchronous copies of the block's
// column indices (into nb1) and walk steps.
template <typename T>
struct Phase0 {
  int64_t r0;
  int nrows, L, S;
  int32_t base, sbase, rs, re, s0, s1;
  int dp, zl;
  V3<T> uni;
};

template <int P>
__device__ __forceinline__ Phase0<typename Prec<P>::T> load_phase0(const MeshView& m, const FieldView& f, int64_t r0) {
  using T = typename Prec<P>::T;
  Phase0<T> p;
  const int R = blockDim.x;
  const int t = threadIdx.x;
  const int64_t r_end = min(r0 + (int64_t)R, m.n);
  p.r0 = r0;
  p.nrows = (int)(r_end - r0);
  p.base = m.row_ptr[r0];
  p.L = m.row_ptr[r_end] - p.base;
  p.sbase = m.walk_ptr[r0];
  p.S = m.walk_ptr[r_end] - p.sbase;
  p.rs = p.re = p.s0 = p.s1 = 0;
  p.dp = p.zl = 0;
  p.uni = V3<T>{T(0), T(0), T(0)};
  const int soff = p.sbase & 3;  // walk bytes are copied as aligned 4-byte words
  if (t < p.nrows) {
    const int64_t i = r0 + t;
    p.rs = m.row_ptr[i];
    p.re = m.row_ptr[i + 1];
    p.s0 = m.walk_ptr[i] - p.sbase + soff;
    p.s1 = m.walk_ptr[i + 1] - p.sbase + soff;
    p.dp = m.diag_pos[i];
    p.uni = load_vec<T>(f.un, i);
    if (p.dp == DIAG_LONG) {  // left to long_rows_kernel: no elements, a zeroed slice
      p.zl = p.re - p.rs;
      p.re = p.rs;
      p.s1 = p.s0;
      p.dp = 0;
    }
  }
  return p;
}

template <bool DEBUG, typename T>
__device__ __forceinline__ void issue_phase0(const MeshView& m, unsigned char* smem, const GatherSmem& lay,
                                             const Phase0<T>& p) {
  const int R = blockDim.x;
  const int t = threadIdx.x;
  if (DEBUG && (p.L > lay.L || p.S > lay.S || R != lay.R)) return;  // reported by stage_records
  int32_t* col = reinterpret_cast<int32_t*>(smem + lay.col());
  uint8_t* walk = smem + lay.walk();
  for (int k = t; k < p.L; k += R) cp_async4(&col[k], m.col_idx + p.base + k);
  const int soff = p.sbase & 3;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(m.walk + (p.sbase - soff));
  const int words = (p.S + soff + 3) >> 2;
  for (int k = t; k < words; k += R) cp_async4(reinterpret_cast<uint32_t*>(walk) + k, src + k);
}

// Phase 1 of a block whose phase-0 copies are in flight: every neighbour's
// record (calculate_transients for the row, asynchronous copies all in
// flight at once), turned into edge vectors d = x_j - x_i (the row's own
// record, its diagonal slot, gives the origin) and velocities in nb0/nb1
// (FP64: scaled by kc = rho/120, the convection weight, once per slot instead
// of once per element step: 3.09 -> 3.02 ms at the 100^3 cube; the float
// walks keep the product in the step, 2% faster there); the accumulators
// zeroed.  Returns false (block-uniform) if the block does not
// fit the layout.
template <int P, bool DEBUG, typename Accum>
__device__ __forceinline__ bool stage_records(const MeshView& m, unsigned char* smem, const GatherSmem& lay,
                                              Accum& acc, const Phase0<typename Prec<P>::T>& p,
                                              BlockRows<typename Prec<P>::T>& b, typename Prec<P>::T kc) {
  using T = typename Prec<P>::T;
  const int R = blockDim.x;
  const int t = threadIdx.x;
  if (DEBUG && (p.L > lay.L || p.S > lay.S || R != lay.R)) {
    if (t == 0) atomicOr(m.err, ERR_STAR);
    return false;
  }
  T4<T>* __restrict__ nb0 = reinterpret_cast<T4<T>*>(smem + lay.nb0());
  T2<T>* __restrict__ nb1 = reinterpret_cast<T2<T>*>(smem + lay.nb1());
  const int32_t* col = reinterpret_cast<const int32_t*>(smem + lay.col());
  cp_async_wait_all();
  __syncthreads();

  const int len = p.re - p.rs;
  const int lb = p.rs - p.base;
  if (t < p.nrows) {
    const unsigned char* recs = static_cast<const unsigned char*>(m.rec);
    constexpr int RB = P == NSI_FP64 ? 64 : 32;
    for (int q = 0, k = t; q < len; ++q, k += R) {
      const int j = col[lb + q];
      if (DEBUG && (j < 0 || j >= m.n)) {
        atomicOr(m.err, ERR_BAD_INDEX);
        continue;
      }
      const unsigned char* r = recs + (size_t)j * RB;
      if constexpr (P == NSI_FP64) {
        cp_async16(&nb0[k], r);
        cp_async16(reinterpret_cast<char*>(&nb0[k]) + 16, r + 16);
        cp_async16(staged_half<P>(smem, lay, k, 0), r + 32);
        cp_async16(staged_half<P>(smem, lay, k, 1), r + 48);
      } else {
        cp_async16(&nb0[k], r);
        cp_async16(staged_half<P>(smem, lay, k, 0), r + 16);
      }
    }
  }
  // every row's column indices have been read: nb1, which holds them, may now
  // be written
  __syncthreads();
  if (t < p.nrows) {
    cp_async_wait_all();
    if (len > 0) {
      const int kd = p.dp * R + t;
      if constexpr (P == NSI_FP64) {
        const T4<T> hi = nb0[kd];
        const V3<T> xi{hi.x, hi.y, hi.z};
        for (int q = 0, k = t; q < len; ++q, k += R) {
          const T4<T> h = nb0[k];
          const T2<T> ua = *static_cast<T2<T>*>(staged_half<P>(smem, lay, k, 0));
          const T2<T> ub = *static_cast<T2<T>*>(staged_half<P>(smem, lay, k, 1));
          nb0[k] = T4<T>{h.x - xi.x, h.y - xi.y, h.z - xi.z, kc * ua.x};
          nb1[k] = T2<T>{kc * ua.y, kc * ub.x};
          acc.zero(k);
        }
      } else {
        const T4<T> hi = nb0[kd];
        const float4 si = *static_cast<float4*>(staged_half<P>(smem, lay, kd, 0));
        const V3<float> xh{hi.x, hi.y, hi.z};
        const V3<float> xl = record_lo(si.z, si.w);
        for (int q = 0, k = t; q < len; ++q, k += R) {
          const T4<T> h = nb0[k];
          const float4 sv = *static_cast<float4*>(staged_half<P>(smem, lay, k, 0));
          const V3<float> d = add(sub(V3<float>{h.x, h.y, h.z}, xh), sub(record_lo(sv.z, sv.w), xl));
          nb0[k] = T4<T>{d.x, d.y, d.z, h.w};
          nb1[k] = T2<T>{sv.x, sv.y};
          acc.zero(k);
        }
      }
    }
  }
  b = BlockRows<T>{R, t, p.nrows, p.L, len, lb, p.s0, p.s1, p.dp, p.r0 + t, p.base, p.uni, p.zl};
  return true;
}

// Phases 0 and 1 of a row-gather block, shared by the full assembly and the
// time-step kernels.
template <int P, bool DEBUG, typename Accum>
__device__ __forceinline__ bool stage_block(const MeshView& m, const FieldView& f, int64_t r0, unsigned char* smem,
                                            const GatherSmem& lay, Accum& acc, BlockRows<typename Prec<P>::T>& b) {
  const Phase0<typename Prec<P>::T> p = load_phase0<P>(m, f, r0);
  issue_phase0<DEBUG>(m, smem, lay, p);
  return stage_records<P, DEBUG>(m, smem, lay, acc, p, b, kc_of<typename Prec<P>::T>(f));
}

// phase 2 of a staged block: every element of each row's star, the diagonal
// and the RHS; ends with a barrier (nb1 and the walk bytes are free after it)
template <int P, bool DEBUG>
__device__ __forceinline__ void gather_compute(const MeshView& m, const FieldView& f, const OutView& o,
                                               unsigned char* smem, const GatherSmem& lay, AccSmem<P>& acc,
                                               const BlockRows<typename Prec<P>::T>& b) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  const int R = b.R, t = b.t, nrows = b.nrows, len = b.len, s0 = b.s0, s1 = b.s1, dp = b.dp;
  const int64_t i = b.i;
  const V3<T> uni = b.uni;
  const T4<T>* __restrict__ nb0 = reinterpret_cast<const T4<T>*>(smem + lay.nb0());
  const T2<T>* __restrict__ nb1 = reinterpret_cast<const T2<T>*>(smem + lay.nb1());
  const uint8_t* walk = smem + lay.walk();
  const T kmu = kmu_of<T>(f);
  const T kc = kc_of<T>(f);
  const T kmass = kmass_of<T>(f);
  Acc<P> detsum;
  detsum.zero();
  if (t < nrows) {
    // phase 2: every element of the row's star, accumulated privately
    if (len > 0) {
      if (DEBUG && dp >= len) atomicOr(m.err, ERR_STAR);
      const int kd = dp * R + t;
      const T4<T> di = nb0[kd];
      const T2<T> ei = nb1[kd];
      const V3<T> u2i{di.w + di.w, ei.x + ei.x, ei.y + ei.y};
      walk_row<P, DEBUG>(walk + s0, s1 - s0, len, nb0, nb1, acc, t, R, u2i, kc, kmu, detsum, m.err);
      // diagonal from the partition of unity (sum_b grad N_b = 0, exact):
      //   A(i,i) = lumped mass - sum_{j != i} A(i,j)   (convection + viscous parts)
      //   G(i,i) = 1/3 sum_{j != i} G(i,j)            (each element adds c_i to three
      //                                                 off-diagonal entries and the diagonal)
      Acc<P> rsum[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) rsum[c].zero();
      acc.row_sums(t, R, len, rsum);  // (the diagonal slot is still zero)
      Acc<P> dg[4];
      if constexpr (P == NSI_MIXED_F32_ACC64) {
        const float p = kmass * detsum.hi;  // kmass * (hi + lo), product error kept
        dg[0].hi = p;
        dg[0].lo = fmaf(kmass, detsum.hi, -p) + kmass * detsum.lo;
        dg[0].add(-rsum[0].hi);
        dg[0].lo -= rsum[0].lo;
#pragma unroll
        for (int c = 1; c < 4; ++c) {  // G: plain float
          dg[c].hi = rsum[c].hi * (1.0f / 3.0f);
          dg[c].lo = 0.f;
        }
      } else {
        dg[0].v = kmass * detsum.v - rsum[0].v;
#pragma unroll
        for (int c = 1; c < 4; ++c) dg[c].v = rsum[c].v * (T(1) / T(3));
      }
      if (!DEBUG || dp < len) acc.set(kd, dg);
    }
    // lumped RHS: (sum_e rho |T_e| / (4 dt)) u^n_i
    const T unk[3] = {uni.x, uni.y, uni.z};
    Out* Rh = static_cast<Out*>(o.rhs);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Acc<P> r;
      const T c = kmass * unk[k];
      if constexpr (P == NSI_MIXED_F32_ACC64) {
        const float p = detsum.hi * c;
        r.hi = p;
        r.lo = fmaf(detsum.hi, c, -p) + detsum.lo * c;
      } else {
        r.v = detsum.v * c;
      }
      store_acc(Rh + k * m.n + i, r);
    }
  }
  __syncthreads();
}

// phase 3 of a block: its contiguous slice of A and G (uses nb0 and acc only)
template <int P>
__device__ __forceinline__ void gather_writeout(const MeshView& m, const OutView& o, unsigned char* smem,
                                                const GatherSmem& lay, AccSmem<P>& acc,
                                                const BlockRows<typename Prec<P>::T>& b) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  const int R = b.R, t = b.t, nrows = b.nrows, L = b.L, len = b.len, lb = b.lb;
  const int32_t base = b.base;
  // phase 3: the block's contiguous slice of A and G.  Every thread moves its
  // own row's finished values into CSR order (nb0 reused as staging), then the
  // block streams the slice out coalesced.
  Out* A = static_cast<Out*>(o.A);
  Out* G = static_cast<Out*>(o.G);
  Out* stage = reinterpret_cast<Out*>(smem + lay.nb0());
  Out* dst[4] = {A + base, G + base, G + m.nnz + base, G + 2 * m.nnz + base};
  if constexpr (sizeof(Out) == sizeof(T4<T>) / 4 || P == NSI_FP64) {
    // room for all four components at once
    if (t < nrows) {
#pragma unroll 4
      for (int q = 0, k = t; q < len; ++q, k += R) {
        const T4<Out> v = acc.values(k);
        stage[lb + q] = v.x;
        stage[L + lb + q] = v.y;
        stage[2 * L + lb + q] = v.z;
        stage[3 * L + lb + q] = v.w;
      }
      for (int q = 0; q < b.zl; ++q)  // a long row: its slice zeroed here, computed later
        stage[lb + q] = stage[L + lb + q] = stage[2 * L + lb + q] = stage[3 * L + lb + q] = Out(0);
    }
    __syncthreads();
    for (int k = t; k < L; k += R) {
      dst[0][k] = stage[k];
      dst[1][k] = stage[L + k];
      dst[2][k] = stage[2 * L + k];
      dst[3][k] = stage[3 * L + k];
    }
  } else {
    // mixed64: one staging round.  Every thread stages its own row's float
    // values in CSR order -- A and G_x, G_y in nb0, G_z in the half of nb1
    // that the next block's column indices (copied in under this write-out by
    // the persistent grid) leave free -- then the block converts them to
    // double exactly and streams them out coalesced (the conversions spread
    // evenly over the threads); an infinite, NaN or subnormal A is converted
    // again by a rare pass.  Last, each row's thread overwrites its diagonal
    // with the double of its compensated pair (leading part in the slot, error
    // term in dlo).
    float* sa = reinterpret_cast<float*>(smem + lay.nb0());
    float* gx = sa + L;
    float* gy = gx + L;
    float* gz = reinterpret_cast<float*>(smem + lay.nb1()) + lay.N();
    if (t < nrows) {
#pragma unroll 4
      for (int q = 0, k = t; q < len; ++q, k += R) {
        const float4 h = acc.hi[k];
        sa[lb + q] = h.w;
        gx[lb + q] = h.x;
        gy[lb + q] = h.y;
        gz[lb + q] = h.z;
      }
      for (int q = 0; q < b.zl; ++q) {  // a long row: its slice zeroed here, computed later
        sa[lb + q] = 0.f;
        gx[lb + q] = gy[lb + q] = gz[lb + q] = 0.f;
      }
    }
    __syncthreads();
    bool slow = false;
    for (int k = t; k < L; k += R) {
      const float a = sa[k];
      slow |= special_float(a);
      dst[0][k] = float_double(a);
      dst[1][k] = float_double(gx[k]);
      dst[2][k] = float_double(gy[k]);
      dst[3][k] = float_double(gz[k]);
    }
    if (__syncthreads_or(slow)) {  // block-uniform and rare
      for (int k = t; k < L; k += R) {
        const float a = sa[k];
        if (special_float(a)) dst[0][k] = nonfinite_bits(a) ? nonfinite_double(a) : (double)a;
      }
      __syncthreads();
    }
    if (t < nrows && len > 0) {
      const float hd = acc.hi[b.dp * R + t].w;
      dst[0][lb + b.dp] = nonfinite_bits(hd) ? nonfinite_double(hd) : pair_double(hd, acc.dlo);
    }
  }
}

// one block of rows [r0, r0 + blockDim.x) of one mesh
template <int P, bool DEBUG>
__device__ __forceinline__ void gather_rows(const MeshView& m, const FieldView& f, const OutView& o, int64_t r0,
                                            unsigned char* smem, const GatherSmem& lay) {
  AccSmem<P> acc(smem + lay.acc(), lay.N());
  BlockRows<typename Prec<P>::T> b;
  if (!stage_block<P, DEBUG>(m, f, r0, smem, lay, acc, b)) return;
  gather_compute<P, DEBUG>(m, f, o, smem, lay, acc, b);
  gather_writeout<P>(m, o, smem, lay, acc, b);
}

// ------------------------------------------- cached-geometry time step ---
// Over time steps on a fixed mesh with fixed rho, mu and dt, the viscous
// part, the lumped mass and the pressure gradient of the assembly do not
// change; only the convection C(u) and the RHS do.  The step kernel forms
//   A = A_static + C(u),  C(i,x) = sum over the star of i of w_e . c_x,
//   w_e = rho/120 (2 u_i + u_p + u_q + u_c)
// and the lumped RHS, where A_static is the A of a full assembly at u = 0
// (the viscous part and the lumped mass).  C has zero row sums (the shape
// gradients of an element sum to zero), so C(i,i) = -sum_{j != i} C(i,j).  G
// is not touched.  The nodal variant forms the paper's per-node outputs
// instead (perform_assembly_in_global_system): rhsid, dt_rho = sum_e
// rho|T|/(4 dt) and mass_rho = sum_e rho|T|/4.  Both follow the element walk
// of the full assembly, with one accumulator per slot (none for the nodal
// outputs).

// A-only accumulator slots, at the stride of the staged record halves (16
// bytes, FP64 two planes of 16): a slot's bytes first receive its record's
// second half, then its accumulator.
template <int P>
struct AccA;
template <>
struct AccA<NSI_MIXED_F32_ACC32> {
  float4* __restrict__ a;
  using Slot = float;
  __device__ __forceinline__ AccA(unsigned char* p) : a(reinterpret_cast<float4*>(p)) {}
  __device__ __forceinline__ void zero(int k) { a[k].x = 0.f; }
  __device__ __forceinline__ Slot load1(int k) const { return a[k].x; }
  __device__ __forceinline__ void store1(int k, Slot v) { a[k].x = v; }
  static __device__ __forceinline__ void add(Slot& s, float x) { s += x; }
  __device__ __forceinline__ void row_sum(int t, int R, int len, Acc<NSI_MIXED_F32_ACC32>& r) const {
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) r.add(a[k].x);
  }
  __device__ __forceinline__ void set(int k, const Acc<NSI_MIXED_F32_ACC32>& r) { a[k].x = r.v; }
};
// mixed64: an off-diagonal entry of C(u) sums the few element terms of its
// edge in plain float (its error term stays zero); the diagonal, minus the
// row's other entries, is the compensated row sum (set() stores the pair).
template <>
struct AccA<NSI_MIXED_F32_ACC64> {
  float4* __restrict__ a;
  using Slot = float2;  // leading part, error term
  __device__ __forceinline__ AccA(unsigned char* p) : a(reinterpret_cast<float4*>(p)) {}
  __device__ __forceinline__ void zero(int k) { a[k].x = a[k].y = 0.f; }
  __device__ __forceinline__ Slot load1(int k) const {
    const float4 v = a[k];
    return make_float2(v.x, v.y);
  }
  __device__ __forceinline__ void store1(int k, Slot v) { reinterpret_cast<float2*>(a + k)[0] = v; }
  static __device__ __forceinline__ void add(Slot& s, float x) { s.x += x; }
  __device__ __forceinline__ void row_sum(int t, int R, int len, Acc<NSI_MIXED_F32_ACC64>& r) const {
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) {
      const float4 v = a[k];
      r.add(v.x);
      r.lo += v.y;
    }
  }
  __device__ __forceinline__ void set(int k, const Acc<NSI_MIXED_F32_ACC64>& r) {
    reinterpret_cast<float2*>(a + k)[0] = make_float2(r.hi, r.lo);
  }
};
template <>
struct AccA<NSI_FP64> {
  T2<double>* __restrict__ a;  // plane 0 of the staged halves
  using Slot = double;
  __device__ __forceinline__ AccA(unsigned char* p) : a(reinterpret_cast<T2<double>*>(p)) {}
  __device__ __forceinline__ void zero(int k) { a[k].x = 0.0; }
  __device__ __forceinline__ Slot load1(int k) const { return a[k].x; }
  __device__ __forceinline__ void store1(int k, Slot v) { a[k].x = v; }
  static __device__ __forceinline__ void add(Slot& s, double x) { s += x; }
  __device__ __forceinline__ void row_sum(int t, int R, int len, Acc<NSI_FP64>& r) const {
#pragma unroll 4
    for (int q = 0, k = t; q < len; ++q, k += R) r.add(a[k].x);
  }
  __device__ __forceinline__ void set(int k, const Acc<NSI_FP64>& r) { a[k].x = r.v; }
};

// The element walk of the time step: det for the lumped sums and, unless
// NODAL, the convection w . c_x into the window's accumulators.  Same window,
// orientation and carried cofactor as walk_row.
template <int P, bool NODAL, bool DEBUG>
__device__ __forceinline__ void walk_step(const uint8_t* __restrict__ st, int nsteps, int len,
                                          const T4<typename Prec<P>::T>* __restrict__ nb0,
                                          const T2<typename Prec<P>::T>* __restrict__ nb1, AccA<P>& acc, int t,
                                          int R, const V3<typename Prec<P>::T>& u2i, typename Prec<P>::T kc,
                                          Acc<P>& detsum, unsigned* err) {
  using T = typename Prec<P>::T;
  using Node = WalkNode<T, typename AccA<P>::Slot>;
  if (nsteps <= 0) return;
  if (DEBUG) {
    bool ok = nsteps >= 3 && !(st[0] & WALK_ELEM) && !(st[1] & WALK_ELEM);
    for (int s = 0; s < nsteps; ++s) ok &= (int)(st[s] & WALK_POS) < len;
    if (!ok) {
      atomicOr(err, ERR_STAR);
      return;
    }
  }
  if (nsteps < 3) return;  // (every walk of a row with elements has at least 3 steps)
  auto load = [&](int k) {
    const T4<T> a = nb0[k];
    Node nd;
    nd.k = k;
    nd.d = V3<T>{a.x, a.y, a.z};
    if constexpr (!NODAL) {
      const T2<T> b = nb1[k];
      nd.u = V3<T>{a.w, b.x, b.y};
      nd.v = acc.load1(k);
    }
    return nd;
  };
  // as walk_row: the two filling steps' nodes loaded directly
  Node p = load((int)(st[0] & WALK_POS) * R + t);
  Node q = load((int)(st[1] & WALK_POS) * R + t);
  V3<T> m = cross(p.d, q.d);
  T sg = T(-1);  // c_c = -sg m
  unsigned w = st[2];
  Node c = load((int)(w & WALK_POS) * R + t);
#pragma unroll 2
  for (int s = 2; s < nsteps; ++s) {
    const unsigned wn = st[min(s + 1, nsteps - 1)];
    const Node cn = load((int)(wn & WALK_POS) * R + t);
    const V3<T> cp = cross(q.d, c.d), cq = cross(c.d, p.d);
    const bool elem = (w & WALK_ELEM) != 0u;
    const T f = elem ? ((w & WALK_NEG) ? T(-1) : T(1)) : T(0);  // orientation, or 0
    detsum.add(f * dot(p.d, cp));
    if constexpr (!NODAL) {
      const V3<T> s3{u2i.x + p.u.x + q.u.x + c.u.x, u2i.y + p.u.y + q.u.y + c.u.y, u2i.z + p.u.z + q.u.z + c.u.z};
      const V3<T> w3 = P == NSI_FP64 ? s3 : V3<T>{kc * s3.x, kc * s3.y, kc * s3.z};
      AccA<P>::add(p.v, f * dot(w3, cp));
      AccA<P>::add(q.v, f * dot(w3, cq));
      AccA<P>::add(c.v, -f * sg * dot(w3, m));
    }
    // as walk_row: the newest node always enters q
    if (w & WALK_EVQ) {
      if constexpr (!NODAL) acc.store1(q.k, q.v);
      m = cq;
      sg = T(1);
    } else {
      if constexpr (!NODAL) acc.store1(p.k, p.v);
      p = q;
      m = cp;
      sg = T(-1);
    }
    q = c;
    c = cn;
    w = wn;
  }
  if constexpr (!NODAL) {
    acc.store1(p.k, p.v);
    acc.store1(q.k, q.v);
  }
}

// outputs of the time-step kernels; kmr = rho/24 (the density mass per det)
struct StepView {
  const void* A_static;
  void* A;
  void* rhs;
  void* dt_rho;
  void* mass_rho;
  double kmr;
  float kmrf;
};

template <typename T, int P>
__device__ __forceinline__ Acc<P> scaled_sum(const Acc<P>& s, T c) {
  Acc<P> r;
  if constexpr (P == NSI_MIXED_F32_ACC64) {
    const float p = s.hi * c;  // c * (hi + lo), product error kept
    r.hi = p;
    r.lo = fmaf(s.hi, c, -p) + s.lo * c;
  } else {
    r.v = s.v * c;
  }
  return r;
}

// one staged block of the time step; `between` runs once the walk is done
// (nb1 and the walk bytes are free) and commits a group of asynchronous
// copies (the persistent grid's next phase 0, or none)
template <int P, bool NODAL, bool DEBUG, typename Hook>
__device__ __forceinline__ void step_block(const MeshView& m, const FieldView& f, const StepView& o,
                                           unsigned char* smem, const GatherSmem& lay, AccA<P>& acc,
                                           const BlockRows<typename Prec<P>::T>& b, const Hook& between) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  const int R = b.R, t = b.t;
  const T4<T>* __restrict__ nb0 = reinterpret_cast<const T4<T>*>(smem + lay.nb0());
  const T2<T>* __restrict__ nb1 = reinterpret_cast<const T2<T>*>(smem + lay.nb1());
  const T kc = kc_of<T>(f);
  const T kmass = kmass_of<T>(f);
  Out* stat = reinterpret_cast<Out*>(smem + lay.stat());
  if constexpr (!NODAL) {
    // the block's slice of A_static, in flight during the walk
    const Out* As = static_cast<const Out*>(o.A_static) + b.base;
    for (int k = t; k < b.L; k += R) {
      if constexpr (sizeof(Out) == 8) cp_async8(stat + k, As + k);
      else cp_async4(stat + k, As + k);
    }
    cp_async_commit();
  }
  Acc<P> detsum;
  detsum.zero();
  if (t < b.nrows) {
    const int kd = b.dp * R + t;
    if (b.len > 0) {
      if (DEBUG && b.dp >= b.len) atomicOr(m.err, ERR_STAR);
      const T4<T> di = nb0[kd];
      const T2<T> ei = nb1[kd];
      const V3<T> u2i{di.w + di.w, ei.x + ei.x, ei.y + ei.y};
      walk_step<P, NODAL, DEBUG>(smem + lay.walk() + b.s0, b.s1 - b.s0, b.len, nb0, nb1, acc, t, R, u2i, kc,
                                 detsum, m.err);
      if constexpr (!NODAL) {  // C(i,i) = -sum_{j != i} C(i,j)
        Acc<P> rsum;
        rsum.zero();
        acc.row_sum(t, R, b.len, rsum);  // (the diagonal slot is still zero)
        Acc<P> dg;
        if constexpr (P == NSI_MIXED_F32_ACC64) {
          dg.hi = -rsum.hi;
          dg.lo = -rsum.lo;
        } else {
          dg.v = -rsum.v;
        }
        if (!DEBUG || b.dp < b.len) acc.set(kd, dg);
      }
    }
    // lumped RHS: (sum_e rho |T_e| / (4 dt)) u^n_i
    const T unk[3] = {b.uni.x, b.uni.y, b.uni.z};
    Out* Rh = static_cast<Out*>(o.rhs);
#pragma unroll
    for (int k = 0; k < 3; ++k) store_acc(Rh + k * m.n + b.i, scaled_sum<T, P>(detsum, kmass * unk[k]));
    if constexpr (NODAL) {
      store_acc(static_cast<Out*>(o.dt_rho) + b.i, scaled_sum<T, P>(detsum, kmass));
      store_acc(static_cast<Out*>(o.mass_rho) + b.i, scaled_sum<T, P>(detsum, (T)(sizeof(T) == 8 ? o.kmr : o.kmrf)));
    }
  }
  __syncthreads();
  between();
  if constexpr (!NODAL) {
    // the block's contiguous slice of A: staged in CSR order, then
    // A = A_static + C streamed out coalesced
    Out* A = static_cast<Out*>(o.A) + b.base;
    cp_async_wait_prior();  // the slice of A_static (the group before `between`'s)
    if constexpr (P == NSI_MIXED_F32_ACC64) {
      float2* stage = reinterpret_cast<float2*>(smem + lay.nb0());
      bool nonfinite = false;  // as in the assembly's write-out
      if (t < b.nrows) {
        for (int q = 0; q < b.len; ++q) {
          const float2 v = acc.load1(q * R + t);
          stage[b.lb + q] = v;
          nonfinite |= nonfinite_bits(v.x);
        }
        // a long row: A_static kept here (C = 0), the convection added later
        for (int q = 0; q < b.zl; ++q) stage[b.lb + q] = make_float2(0.f, 0.f);
      }
      const bool fix = __syncthreads_or(nonfinite);
#pragma unroll 2
      for (int k = t; k < b.L; k += R) A[k] = stat[k] + pair_double(stage[k].x, stage[k].y);
      if (fix)
        for (int k = t; k < b.L; k += R)
          if (nonfinite_bits(stage[k].x)) A[k] = stat[k] + nonfinite_double(stage[k].x);
    } else {
      Out* stage = reinterpret_cast<Out*>(smem + lay.nb0());
      if (t < b.nrows) {
        for (int q = 0; q < b.len; ++q) stage[b.lb + q] = acc.load1(q * R + t);
        for (int q = 0; q < b.zl; ++q) stage[b.lb + q] = Out(0);  // a long row (as above)
      }
      __syncthreads();
#pragma unroll 2
      for (int k = t; k < b.L; k += R) A[k] = stat[k] + stage[k];
    }
  }
}

template <int P, bool NODAL, bool DEBUG>
__global__ void __launch_bounds__(128) step_kernel(MeshView m, FieldView f, StepView o, GatherSmem lay) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AccA<P> acc(smem_raw + lay.acc());
  BlockRows<typename Prec<P>::T> b;
  if (!stage_block<P, DEBUG>(m, f, (int64_t)blockIdx.x * blockDim.x, smem_raw, lay, acc, b)) return;
  step_block<P, NODAL, DEBUG>(m, f, o, smem_raw, lay, acc, b, []() { cp_async_commit(); });
}

// the time step as a persistent grid: a CTA's next block starts its phase-0
// copies (column indices into nb1, walk bytes) under the current block's
// write-out, as in gather_persistent_kernel
template <int P, bool NODAL, bool DEBUG>
__global__ void __launch_bounds__(128) step_persistent_kernel(MeshView m, FieldView f, StepView o, GatherSmem lay,
                                                              int64_t nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using T = typename Prec<P>::T;
  int64_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  const int R = blockDim.x;
  AccA<P> acc(smem_raw + lay.acc());
  Phase0<T> p = load_phase0<P>(m, f, blk * R);
  issue_phase0<DEBUG>(m, smem_raw, lay, p);
  while (true) {
    BlockRows<T> b;
    if (!stage_records<P, DEBUG>(m, smem_raw, lay, acc, p, b, kc_of<T>(f))) return;
    const int64_t nxt = blk + gridDim.x;
    const bool more = nxt < nblocks;  // block-uniform
    Phase0<T> pn = p;
    if (more) pn = load_phase0<P>(m, f, nxt * R);
    step_block<P, NODAL, DEBUG>(m, f, o, smem_raw, lay, acc, b, [&]() {
      if (more) issue_phase0<DEBUG>(m, smem_raw, lay, pn);
      cp_async_commit();
    });
    if (!more) return;
    blk = nxt;
    p = pn;
  }
}

// ------------------------------------------------ badly shaped elements ---
// Rows listed at create (mixed modes: the rows of the nodes of an element with
// |d1||d2||d3| > EXACT_RATIO |det|) are recomputed after the assembly with
// every element of their star evaluated in double from the coordinates
// (leading + residual float parts) and velocities, and their entries
// overwritten: a float determinant of such an element would carry about that
// ratio times the float rounding of its edge vectors.  One thread per row,
// its sums in a local array.  MODE 0: A, G and rhs; 1: rhs only (the time
// step: the convection does not involve the determinant); 2: rhs, dt_rho and
// mass_rho.
template <int P, int MODE>
__global__ void __launch_bounds__(64) exact_rows_kernel(MeshView m, FieldView f, void* A, void* G, void* rhs,
                                                        void* dt_rho, void* mass_rho, double kmr, const int32_t* rows,
                                                        const int32_t* ptr, const uint32_t* inc, int64_t count) {
  using Out = typename Prec<P>::Out;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int64_t i = rows[r];
  const int32_t rs = m.row_ptr[i], len = m.row_ptr[i + 1] - rs;
  if (len > STAR_MAX_ROW) return;
  const int32_t* cols = m.col_idx + rs;
  auto coord = [&](int64_t j) {
    const float4 h = m.xyz_hi[j], l = m.xyz_lo[j];
    return V3<double>{(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
  };
  auto vel = [&](int64_t j) {
    const V3<float> u = load_vec<float>(f.u, j);
    return V3<double>{u.x, u.y, u.z};
  };
  // even permutations of (0,1,2,3) that bring vertex a to the front
  const int EVEN[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
  double acc[STAR_MAX_ROW][4];
  for (int q = 0; q < len; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0;
  const V3<double> xi = coord(i), ui = vel(i);
  double detsum = 0.0;
  int dpos = 0;
  for (int q = 0; q < len; ++q)
    if (cols[q] == i) dpos = q;
  for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) {
    const int64_t e = inc[t] >> 2;
    const int a = (int)(inc[t] & 3u);
    const int4 v4 = m.lnods[e];
    const int v[4] = {v4.x, v4.y, v4.z, v4.w};
    int pos[3];
    V3<double> d[3], u[3];
    for (int b = 0; b < 3; ++b) {
      const int j = v[EVEN[a][b]];
      int lo = 0, hi = len - 1;  // position of j in the row (columns ascending)
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      pos[b] = lo;
      d[b] = sub(coord(j), xi);
      u[b] = vel(j);
    }
    const V3<double> c[3] = {cross(d[1], d[2]), cross(d[2], d[0]), cross(d[0], d[1])};
    const double det = dot(d[0], c[0]);
    const V3<double> ci{-(c[0].x + c[1].x + c[2].x), -(c[0].y + c[1].y + c[2].y), -(c[0].z + c[1].z + c[2].z)};
    const double kv = f.kmu / det;
    const V3<double> w3{f.kc * (2.0 * ui.x + u[0].x + u[1].x + u[2].x) + kv * ci.x,
                        f.kc * (2.0 * ui.y + u[0].y + u[1].y + u[2].y) + kv * ci.y,
                        f.kc * (2.0 * ui.z + u[0].z + u[1].z + u[2].z) + kv * ci.z};
    for (int b = 0; b < 3; ++b) {
      acc[pos[b]][0] += dot(w3, c[b]);
      acc[pos[b]][1] += ci.x;
      acc[pos[b]][2] += ci.y;
      acc[pos[b]][3] += ci.z;
    }
    detsum += det;
  }
  // lumped RHS and nodal sums
  const V3<double> un = [&] {
    if constexpr (P == NSI_FP64) return load_vec<double>(f.un, i);
    else {
      const V3<float> w = load_vec<float>(f.un, i);
      return V3<double>{w.x, w.y, w.z};
    }
  }();
  Out* Rh = static_cast<Out*>(rhs);
  Rh[i] = (Out)(f.kmass * detsum * un.x);
  Rh[m.n + i] = (Out)(f.kmass * detsum * un.y);
  Rh[2 * m.n + i] = (Out)(f.kmass * detsum * un.z);
  if constexpr (MODE == 2) {
    static_cast<Out*>(dt_rho)[i] = (Out)(f.kmass * detsum);
    static_cast<Out*>(mass_rho)[i] = (Out)(kmr * detsum);
  }
  if constexpr (MODE == 0) {
    // diagonal from the partition of unity, as in the row gather
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < len; ++q)
      if (q != dpos)
        for (int k = 0; k < 4; ++k) s[k] += acc[q][k];
    acc[dpos][0] = f.kmass * detsum - s[0];
    for (int k = 1; k < 4; ++k) acc[dpos][k] = s[k] / 3.0;
    Out* Ao = static_cast<Out*>(A) + rs;
    Out* Go = static_cast<Out*>(G) + rs;
    for (int q = 0; q < len; ++q) {
      Ao[q] = (Out)acc[q][0];
      for (int d = 0; d < 3; ++d) Go[d * m.nnz + q] = (Out)(-acc[q][d + 1] / 24.0);
    }
  }
}

// ---------------------------------------------------------- long rows ---
// Rows the row gather leaves out (more than 32 entries, whose row positions
// do not fit the walk's five bits, or a star the walk encoder could not
// cover), computed after the kernels by one thread per row, in double (the
// coordinates of the handle's copy, the velocities as given): every
// off-diagonal entry (i, j) sums the contributions of the row's elements that
// contain j, w . c_j and -c_i / 24 (with i first and the element's other
// nodes in an even order, so that det > 0); the diagonal follows from the
// partition of unity as in the row gather, A(i,i) = lumped mass - sum_{j != i}
// A(i,j) and G(i,i) = 1/3 sum_{j != i} G(i,j).  MODE 0: A, G and rhs; 1: the
// time step, A = A_static + C(u) (A may alias A_static: each entry is read
// before it is written, by this thread) and rhs; 2: rhs, dt_rho and
// mass_rho.  The row's elements are scanned once per entry: the rows are few.
template <int P, int MODE>
__global__ void __launch_bounds__(64) long_rows_kernel(MeshView m, FieldView f, const void* A_static, void* A,
                                                       void* G, void* rhs, void* dt_rho, void* mass_rho, double kmr,
                                                       const int32_t* rows, const int32_t* ptr, const uint32_t* inc,
                                                       int64_t count) {
  using Out = typename Prec<P>::Out;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int64_t i = rows[r];
  const int32_t rs = m.row_ptr[i], len = m.row_ptr[i + 1] - rs;
  const int32_t* cols = m.col_idx + rs;
  auto coord = [&](int64_t j) {
    if constexpr (P == NSI_FP64) {
      const D4 x = m.xyz64[j];
      return V3<double>{x.x, x.y, x.z};
    } else {
      const float4 h = m.xyz_hi[j], l = m.xyz_lo[j];
      return V3<double>{(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
    }
  };
  auto vel = [&](const void* const* comp, int64_t j) {
    if constexpr (P == NSI_FP64) return load_vec<double>(comp, j);
    else {
      const V3<float> w = load_vec<float>(comp, j);
      return V3<double>{w.x, w.y, w.z};
    }
  };
  // even permutations of (0,1,2,3) that bring vertex a to the front
  const int EVEN[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
  const V3<double> xi = coord(i), ui = vel(f.u, i);
  // one element of the row: its other nodes in even order, their edge vectors
  // from node i, cofactors c[0..2] = det(J) grad N of those nodes, c_i, det
  struct El {
    int v[3];
    V3<double> c[3], ci;
    double det;
    V3<double> w;  // rho/120 (2 u_i + sum of the others) + (MODE 0) mu/(6 det) c_i
  };
  auto element = [&](int32_t t) {
    El el;
    const int64_t e = inc[t] >> 2;
    const int a = (int)(inc[t] & 3u);
    const int4 v4 = m.lnods[e];
    const int v[4] = {v4.x, v4.y, v4.z, v4.w};
    V3<double> d[3], us{2.0 * ui.x, 2.0 * ui.y, 2.0 * ui.z};
    for (int b = 0; b < 3; ++b) {
      el.v[b] = v[EVEN[a][b]];
      d[b] = sub(coord(el.v[b]), xi);
      us = add(us, vel(f.u, el.v[b]));
    }
    el.c[0] = cross(d[1], d[2]);
    el.c[1] = cross(d[2], d[0]);
    el.c[2] = cross(d[0], d[1]);
    el.det = dot(d[0], el.c[0]);
    el.ci = V3<double>{-(el.c[0].x + el.c[1].x + el.c[2].x), -(el.c[0].y + el.c[1].y + el.c[2].y),
                       -(el.c[0].z + el.c[1].z + el.c[2].z)};
    const double kv = MODE == 0 ? f.kmu / el.det : 0.0;
    el.w = V3<double>{f.kc * us.x + kv * el.ci.x, f.kc * us.y + kv * el.ci.y, f.kc * us.z + kv * el.ci.z};
    return el;
  };
  double detsum = 0.0;
  for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) detsum += element(t).det;
  if constexpr (MODE != 2) {
    Out* Ao = static_cast<Out*>(A) + rs;
    const Out* As = MODE == 1 ? static_cast<const Out*>(A_static) + rs : nullptr;
    Out* Go = MODE == 0 ? static_cast<Out*>(G) + rs : nullptr;
    double sa = 0.0, sg[3] = {0.0, 0.0, 0.0};
    int dpos = 0;
    for (int q = 0; q < len; ++q) {
      const int32_t j = cols[q];
      if (j == i) {
        dpos = q;
        continue;
      }
      double a = 0.0, g[3] = {0.0, 0.0, 0.0};
      for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) {
        const int4 v4 = m.lnods[inc[t] >> 2];
        if (v4.x != j && v4.y != j && v4.z != j && v4.w != j) continue;
        const El el = element(t);
        const int b = el.v[0] == j ? 0 : el.v[1] == j ? 1 : 2;
        a += dot(el.w, el.c[b]);
        g[0] += el.ci.x;
        g[1] += el.ci.y;
        g[2] += el.ci.z;
      }
      sa += a;
      if constexpr (MODE == 0) {
        Ao[q] = (Out)a;
        for (int d = 0; d < 3; ++d) {
          Go[d * m.nnz + q] = (Out)(-g[d] / 24.0);
          sg[d] += g[d];
        }
      } else {
        Ao[q] = (Out)((double)As[q] + a);
      }
    }
    if (len > 0) {
      if constexpr (MODE == 0) {
        Ao[dpos] = (Out)(f.kmass * detsum - sa);
        for (int d = 0; d < 3; ++d) Go[d * m.nnz + dpos] = (Out)(-sg[d] / 72.0);
      } else {
        Ao[dpos] = (Out)((double)As[dpos] - sa);
      }
    }
  }
  const V3<double> un = vel(f.un, i);
  Out* Rh = static_cast<Out*>(rhs);
  Rh[i] = (Out)(f.kmass * detsum * un.x);
  Rh[m.n + i] = (Out)(f.kmass * detsum * un.y);
  Rh[2 * m.n + i] = (Out)(f.kmass * detsum * un.z);
  if constexpr (MODE == 2) {
    static_cast<Out*>(dt_rho)[i] = (Out)(f.kmass * detsum);
    static_cast<Out*>(mass_rho)[i] = (Out)(kmr * detsum);
  }
}

// ------------------------------------------------------ edge-fan kernel ---
// One thread per CSR entry (i, j) of a block of whole rows.  An off-diagonal
// entry walks the ring of nodes k_0 .. k_{r-1} around the edge (i, j): the
// elements containing the edge are (i, j, k_m, k_{m+1}), positively oriented.
// With i as the origin and q_m = d_j x d_{k_m}, such an element has
//   c_j = d_{k_m} x d_{k_{m+1}},  c_i = -(c_j + q_m - q_{m+1}),  det = d_j . c_j
// (c_{k_m} = -q_{m+1} and c_{k_{m+1}} = q_m come for free from the ring), and
// adds w . c_j to A(i, j), c_i to the pressure-gradient sum and det to the
// lumped mass sum, with w = rho/120 (2 u_i + u_j + u_{k_m} + u_{k_{m+1}}) +
// mu/(6 det) c_i.  All sums stay in registers.  The diagonal entry receives
// the row totals through a tree reduction in shared memory:
//   A(i,i) = M_i - sum_{j != i} A(i,j), G(i,i) = 1/3 sum_{j != i} G(i,j),
//   M_i = rho/(24 dt) * 1/3 sum_{j != i} sum_fan det
// (every element of the star appears in the fans of its three other nodes).
// Every thread then writes its own entry: the block's slice of A and G goes
// out coalesced.

// shared-memory layout of a fan block (T entries)
template <int P>
struct FanSmem {
  using T = typename Prec<P>::T;
  static constexpr size_t rec() { return 0; }                                        // T4 [T] x 2
  static constexpr size_t rp(int Tn) { return 2 * sizeof(T4<T>) * (size_t)Tn; }      // int32 [T + 1]
  static constexpr size_t red(int Tn) { return rp(Tn) + (((size_t)4 * (Tn + 1) + 15) & ~size_t(15)); }
  static constexpr size_t total(int Tn) { return red(Tn) + 5 * sizeof(Acc<P>) * (size_t)Tn; }
};

template <int P>
__device__ __forceinline__ void acc_merge(Acc<P>& a, const Acc<P>& b) {
  if constexpr (P == NSI_MIXED_F32_ACC64) {
    a.add(b.hi);
    a.lo += b.lo;
  } else {
    a.v += b.v;
  }
}

// x / 3 of an accumulator (compensated for the pair)
template <int P>
__device__ __forceinline__ Acc<P> acc_third(const Acc<P>& a) {
  Acc<P> r;
  if constexpr (P == NSI_MIXED_F32_ACC64) {
    const float q = a.hi * (1.0f / 3.0f);
    r.hi = q;
    r.lo = fmaf(a.hi, 1.0f / 3.0f, -q) + a.lo * (1.0f / 3.0f);
  } else {
    r.v = a.v * (typename Prec<P>::T(1) / typename Prec<P>::T(3));
  }
  return r;
}

// c * (a), product error kept for the pair
template <int P>
__device__ __forceinline__ Acc<P> acc_scale(const Acc<P>& a, typename Prec<P>::T c) {
  Acc<P> r;
  if constexpr (P == NSI_MIXED_F32_ACC64) {
    const float p = c * a.hi;
    r.hi = p;
    r.lo = fmaf(c, a.hi, -p) + c * a.lo;
  } else {
    r.v = c * a.v;
  }
  return r;
}

// One CSR entry of a fan block (blocks of whole rows, one thread per entry):
// its row within the block, the row's start and length in the block, the
// diagonal's position, the fan word, and (node i the row's node, j the
// column's) the edge vector d_j = x_j - x_i and the velocities u_j, u_i.
template <typename T>
struct FanEntry {
  int64_t R0;
  int32_t base;
  int nr, L, row, a, len, dp;
  uint32_t w;
  V3<T> dj, uj, ui;
};

// Steps 1-2 of a fan block: the row starts of the block, this entry's
// neighbour record (calculate_transients), its row and edge vector; then
// every entry's record in shared memory is replaced by (edge vector from its
// row's node, velocity).  Returns false (block-uniform) when DEBUG finds the
// block larger than the kernel's.
template <int P, bool DEBUG>
__device__ __forceinline__ bool fan_entry(const MeshView& m, int64_t blk, T4<typename Prec<P>::T>* rec0,
                                          T4<typename Prec<P>::T>* rec1, int32_t* rp,
                                          FanEntry<typename Prec<P>::T>& e) {
  using T = typename Prec<P>::T;
  constexpr int TB = FAN_BLOCK;
  const int k = threadIdx.x;
  e.R0 = m.fan_blk[blk];
  const int64_t R1 = m.fan_blk[blk + 1];
  e.nr = (int)(R1 - e.R0);
  e.base = m.row_ptr[e.R0];
  e.L = m.row_ptr[R1] - e.base;
  if (DEBUG && (e.L > TB || e.nr > TB)) {
    if (k == 0) atomicOr(m.err, ERR_STAR);
    return false;
  }
  for (int r = k; r <= e.nr; r += TB) rp[r] = m.row_ptr[e.R0 + r] - e.base;
  e.w = 0;
  if (k < e.L) {
    const int j = m.col_idx[e.base + k];
    e.w = m.fan[e.base + k];
    if (!DEBUG || (j >= 0 && j < m.n)) {
      const unsigned char* r = static_cast<const unsigned char*>(m.rec) + (size_t)j * (2 * sizeof(T4<T>));
      if constexpr (P == NSI_FP64) {
        cp_async16(&rec0[k], r);
        cp_async16(reinterpret_cast<char*>(&rec0[k]) + 16, r + 16);
        cp_async16(&rec1[k], r + 32);
        cp_async16(reinterpret_cast<char*>(&rec1[k]) + 16, r + 48);
      } else {
        cp_async16(&rec0[k], r);
        cp_async16(&rec1[k], r + 16);
      }
    } else {
      atomicOr(m.err, ERR_BAD_INDEX);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  e.row = e.a = e.len = e.dp = 0;
  e.dj = e.uj = e.ui = V3<T>{T(0), T(0), T(0)};
  if (k < e.L) {
    int lo = 0, hi = e.nr - 1;  // last row whose start is <= k
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= k) lo = mid;
      else hi = mid - 1;
    }
    e.row = lo;
    e.a = rp[e.row];
    e.len = rp[e.row + 1] - e.a;
    e.dp = m.diag_pos[e.R0 + e.row];
    const T4<T> h = rec0[k], s = rec1[k];
    const T4<T> hd = rec0[e.a + e.dp], sd = rec1[e.a + e.dp];
    if constexpr (P == NSI_FP64) {
      e.dj = {h.x - hd.x, h.y - hd.y, h.z - hd.z};
      e.uj = {s.x, s.y, s.z};
      e.ui = {sd.x, sd.y, sd.z};
    } else {
      const V3<float> lj = record_lo(s.z, s.w), li = record_lo(sd.z, sd.w);
      e.dj = add(sub(V3<float>{h.x, h.y, h.z}, V3<float>{hd.x, hd.y, hd.z}), sub(lj, li));
      e.uj = {h.w, s.x, s.y};
      e.ui = {hd.w, sd.x, sd.y};
    }
  }
  __syncthreads();
  if (k < e.L) {
    rec0[k] = T4<T>{e.dj.x, e.dj.y, e.dj.z, T(0)};
    rec1[k] = T4<T>{e.uj.x, e.uj.y, e.uj.z, T(0)};
  }
  __syncthreads();
  return true;
}

template <int P, bool DEBUG>
__device__ __forceinline__ void fan_block(const MeshView& m, const FieldView& f, const OutView& o, int64_t blk,
                                          unsigned char* smem) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  constexpr int TB = FAN_BLOCK;
  T4<T>* rec0 = reinterpret_cast<T4<T>*>(smem + FanSmem<P>::rec());
  T4<T>* rec1 = rec0 + TB;
  int32_t* rp = reinterpret_cast<int32_t*>(smem + FanSmem<P>::rp(TB));
  Acc<P>* red = reinterpret_cast<Acc<P>*>(smem + FanSmem<P>::red(TB));  // 5 arrays of TB
  const int k = threadIdx.x;
  FanEntry<T> fe;
  if (!fan_entry<P, DEBUG>(m, blk, rec0, rec1, rp, fe)) return;
  const int64_t R0 = fe.R0;
  const int nr = fe.nr, L = fe.L, row = fe.row, a = fe.a, len = fe.len, dp = fe.dp;
  const int32_t base = fe.base;
  const uint32_t w = fe.w;
  const V3<T> dj = fe.dj, uj = fe.uj, ui = fe.ui;
  const T kc = kc_of<T>(f), kmu = kmu_of<T>(f), kmass = kmass_of<T>(f);
  const T kg = (T)(-1.0 / 24.0);

  // 3. the fan of an off-diagonal entry, summed in registers
  Acc<P> sA, sGx, sGy, sGz, sD;
  sA.zero(); sGx.zero(); sGy.zero(); sGz.zero(); sD.zero();
  const int nring = (w >> 24) & 7;
  if (k < L && nring > 0) {
    const bool closed = (w >> 27) & 1;
    const int nel = closed ? nring : nring - 1;
    const V3<T> uij{ui.x + ui.x + uj.x, ui.y + ui.y + uj.y, ui.z + ui.z + uj.z};  // 2 u_i + u_j
    auto node = [&](int mpos, V3<T>& d, V3<T>& u) {
      const int pos = (w >> (4 * mpos)) & 15;
      if (DEBUG && pos >= len) atomicOr(m.err, ERR_STAR);
      const T4<T> x = rec0[a + pos], y = rec1[a + pos];
      d = {x.x, x.y, x.z};
      u = {y.x, y.y, y.z};
    };
    V3<T> d0, u0;
    node(0, d0, u0);
    V3<T> q0 = cross(dj, d0);
    const V3<T> dfirst = d0, ufirst = u0, qfirst = q0;
    for (int e = 0; e < nel; ++e) {
      V3<T> d1, u1, q1;
      if (e + 1 < nring) {
        node(e + 1, d1, u1);
        q1 = cross(dj, d1);
      } else {  // closing element of an interior ring
        d1 = dfirst;
        u1 = ufirst;
        q1 = qfirst;
      }
      const V3<T> cj = cross(d0, d1);
      const T det = dot(dj, cj);
      const V3<T> ci{-(cj.x + q0.x - q1.x), -(cj.y + q0.y - q1.y), -(cj.z + q0.z - q1.z)};
      const T kv = kmu * rcp_fast(det);
      const V3<T> w3{kc * (uij.x + u0.x + u1.x) + kv * ci.x, kc * (uij.y + u0.y + u1.y) + kv * ci.y,
                     kc * (uij.z + u0.z + u1.z) + kv * ci.z};
      sA.add(dot(w3, cj));
      sGx.add(ci.x);
      sGy.add(ci.y);
      sGz.add(ci.z);
      sD.add(det);
      d0 = d1;
      u0 = u1;
      q0 = q1;
    }
  }

  // 4. row totals for the diagonal: tree reduction over each row's entries
  Acc<P>* rA = red;
  Acc<P>* rGx = red + TB;
  Acc<P>* rGy = red + 2 * TB;
  Acc<P>* rGz = red + 3 * TB;
  Acc<P>* rD = red + 4 * TB;
  if (k < L) {
    rA[k] = sA;
    rGx[k] = sGx;
    rGy[k] = sGy;
    rGz[k] = sGz;
    rD[k] = sD;
  }
  __syncthreads();
#pragma unroll
  for (int st = 1; st < FAN_MAX_ROW; st <<= 1) {
    if (k < L && ((k - a) & (2 * st - 1)) == 0 && k - a + st < len) {
      acc_merge<P>(rA[k], rA[k + st]);
      acc_merge<P>(rGx[k], rGx[k + st]);
      acc_merge<P>(rGy[k], rGy[k + st]);
      acc_merge<P>(rGz[k], rGz[k + st]);
      acc_merge<P>(rD[k], rD[k + st]);
    }
    __syncthreads();
  }

  // 5. this entry's outputs (coalesced across the block), the diagonal's and the RHS
  Out* A = static_cast<Out*>(o.A);
  Out* G = static_cast<Out*>(o.G);
  Out* Rh = static_cast<Out*>(o.rhs);
  if (k < L) {
    const int64_t g = (int64_t)base + k;
    if (k == a + dp) {
      const Acc<P> d3 = acc_third<P>(rD[a]);
      const Acc<P> mass = acc_scale<P>(d3, kmass);
      Acc<P> add_ = mass;
      if constexpr (P == NSI_MIXED_F32_ACC64) {
        add_.add(-rA[a].hi);
        add_.lo -= rA[a].lo;
      } else {
        add_.v = mass.v - rA[a].v;
      }
      store_acc(A + g, add_);
      store_acc(G + g, acc_scale<P>(acc_third<P>(rGx[a]), kg));
      store_acc(G + m.nnz + g, acc_scale<P>(acc_third<P>(rGy[a]), kg));
      store_acc(G + 2 * m.nnz + g, acc_scale<P>(acc_third<P>(rGz[a]), kg));
      const int64_t i = R0 + row;
      const V3<T> un = load_vec<T>(f.un, i);
      store_acc(Rh + i, acc_scale<P>(mass, un.x));
      store_acc(Rh + m.n + i, acc_scale<P>(mass, un.y));
      store_acc(Rh + 2 * m.n + i, acc_scale<P>(mass, un.z));
    } else {
      store_acc(A + g, sA);
      store_acc(G + g, acc_scale<P>(sGx, kg));
      store_acc(G + m.nnz + g, acc_scale<P>(sGy, kg));
      store_acc(G + 2 * m.nnz + g, acc_scale<P>(sGz, kg));
    }
  }
  // rows without entries (nodes in no element): zero right-hand side
  for (int r = k; r < nr; r += TB) {
    if (rp[r + 1] == rp[r]) {
      Acc<P> z;
      z.zero();
      store_acc(Rh + R0 + r, z);
      store_acc(Rh + m.n + R0 + r, z);
      store_acc(Rh + 2 * m.n + R0 + r, z);
    }
  }
}

template <int P, bool DEBUG>
__global__ void __launch_bounds__(FAN_BLOCK) fan_kernel(MeshView m, FieldView f, OutView o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fan_block<P, DEBUG>(m, f, o, blockIdx.x, smem_raw);
}

// --------------------------------------------- stabilised velocity block ---
// The paper's 12x12 element matrix (Section II-A: every pair of dimensions of
// two nodes coupled, equal dimensions receiving the scalar part) assembled on
// the CSR pattern as one 3x3 block per entry, Auu[(3 a + b) nnz + p] the
// (a, b) entry of the block of entry p = (i, j):
//   Auu(i,j)[a][b] = delta_ab (A(i,j) + S(i,j)) + K(i,j)[a][b]
// with A the Galerkin operator and the implicit terms of Codina's algebraic
// subgrid scales (Comput. Methods Appl. Mech. Engrg. 191 (2002) 4295-4321,
// linear elements, c1 = 4, c2 = 2):
//   tau1 = (4 mu / h^2 + 2 rho |ubar| / h)^-1,  tau2 = h^2 / (4 tau1),
//   S(i,j)       += tau1 rho^2 int (u . grad N_i)(u . grad N_j)
//   K(i,j)[a][b] += mu int d_b N_i d_a N_j + tau2 int d_a N_i d_b N_j
// per element, h = (6 |T|)^(1/3) = det^(1/3), ubar the mean of the element's
// four node velocities.  With the cofactors c_n = det grad N_n, the sum us of
// the four velocities and s = |us| (so 2 rho |ubar| h = rho s h / 2, and the
// moments int lam_m lam_n = |T| (1 + delta_mn) / 20 of the linear velocity):
//   S += rho^2 / (120 h (4 mu + rho s h / 2)) [(us . c_i)(us . c_j) + sum_n (u_n . c_i)(u_n . c_j)]
//   K[a][b] += kv c_j[a] c_i[b] + kd c_i[a] c_j[b],
//   kv = mu / (6 det),  kd = tau2 / (6 det) = kv + rho s h / (48 det).
// Every term vanishes on a constant column field (sum_n c_n = 0), so, as for
// A, the diagonal block is the lumped mass times I minus the sum of the row's
// off-diagonal blocks.
struct StabConst {
  double ks, k4mu, krh, kr48;  // rho^2 / 120, 4 mu, rho / 2, rho / 48
  float ksf, k4muf, krhf, kr48f;
};

static StabConst stab_const(const NsiFields* f) {
  StabConst c;
  c.ks = f->rho * f->rho / 120.0;
  c.k4mu = 4.0 * f->mu;
  c.krh = f->rho / 2.0;
  c.kr48 = f->rho / 48.0;
  c.ksf = (float)c.ks;
  c.k4muf = (float)c.k4mu;
  c.krhf = (float)c.krh;
  c.kr48f = (float)c.kr48;
  return c;
}

template <typename T>
struct StabK {
  T ks, k4mu, krh, kr48;
};
template <typename T>
__device__ __forceinline__ StabK<T> stab_k(const StabConst& c) {
  if constexpr (sizeof(T) == 8) return StabK<T>{c.ks, c.k4mu, c.krh, c.kr48};
  else return StabK<T>{c.ksf, c.k4muf, c.krhf, c.kr48f};
}
__device__ __forceinline__ float cbrt_of(float x) { return cbrtf(x); }
__device__ __forceinline__ double cbrt_of(double x) { return cbrt(x); }
__device__ __forceinline__ float sqrt_of(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_of(double x) { return sqrt(x); }
__device__ __forceinline__ float fma_of(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_of(double a, double b, double c) { return fma(a, b, c); }

// One element's stabilisation terms for the entry (row node, column node):
// ci, cj the two nodes' cofactors, det, and the element's four node
// velocities (any order).  K is added to; S is returned.
template <typename T>
__device__ __forceinline__ T stab_terms(const V3<T>& ci, const V3<T>& cj, T det, const V3<T>& ua, const V3<T>& ub,
                                        const V3<T>& uc, const V3<T>& ud, const StabK<T>& k, T kmu, T (&K)[9]) {
  const V3<T> us = add(add(ua, ub), add(uc, ud));
  const T h = cbrt_of(det);
  const T sh = sqrt_of(dot(us, us)) * h;  // s h
  const T rdet = rcp_fast(det);
  T mm = dot(us, ci) * dot(us, cj);
  mm = fma_of(dot(ua, ci), dot(ua, cj), mm);
  mm = fma_of(dot(ub, ci), dot(ub, cj), mm);
  mm = fma_of(dot(uc, ci), dot(uc, cj), mm);
  mm = fma_of(dot(ud, ci), dot(ud, cj), mm);
  const T kv = kmu * rdet;
  const T kd = fma_of(k.kr48 * sh, rdet, kv);
  const T r[3] = {ci.x, ci.y, ci.z}, c[3] = {cj.x, cj.y, cj.z};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) K[3 * a + b] = fma_of(kv * c[a], r[b], fma_of(kd * r[a], c[b], K[3 * a + b]));
  return k.ks * mm * rcp_fast(h * fma_of(k.krh, sh, k.k4mu));
}

// Lengths of Codina's tau for one element: h = det^(1/3) and s h with s the
// norm of the four velocities' sum.  Float: h from the exp2/log2 estimate and
// one Newton step for the cube root (h <- (2 h + det / h^2) / 3), s as
// s2 rsqrt(s2) (0 for s2 = 0); double: cbrt and sqrt.
__device__ __forceinline__ void tau_lengths(float det, float s2, float& h, float& sh) {
  const float h0 = exp2f(__log2f(det) * (1.0f / 3.0f));
  h = fmaf(h0, 2.0f / 3.0f, det * __fdividef(1.0f / 3.0f, h0 * h0));
  sh = (s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f) * h;
}
__device__ __forceinline__ void tau_lengths(double det, double s2, double& h, double& sh) {
  h = cbrt(det);
  sh = sqrt(s2) * h;
}

// Shared memory of one warp of the stabilised row kernel: entry records
// (component-major [6][32]: edge vector from the row's node, velocity), then
// element records for a chunk of 64 elements (element-major, five T4 each:
// (c_i, mu/(6 det)), (c_1, A+S to node 1), (c_2, ..), (c_3, ..),
// (tau2/(6 det), det, -, -)), then per entry three 64-bit masks of the
// chunk's elements holding the entry as their first, second or third node.
template <int P>
struct StarSmem {
  using T = typename Prec<P>::T;
  static constexpr int CHUNK = 64;
  static constexpr size_t ent() { return 0; }
  static constexpr size_t el() { return sizeof(T) * 6 * 32; }
  static constexpr size_t mask() { return el() + sizeof(T4<T>) * 5 * CHUNK; }
  static constexpr size_t bytes() { return mask() + sizeof(unsigned) * 6 * 32; }
};
constexpr int STAR_WARPS = 4;  // warps (tasks) per block

// The stabilised block by rows, one warp per task (one row of up to 32
// entries, or two consecutive rows of up to 16 on the two half-warps).
//  1. Each entry lane loads its column's node record; the edge vector from the
//     row's node (the diagonal lane's record, by shuffles) and the velocity go
//     to shared memory.
//  2. In chunks of 64 elements (two per lane), each lane takes elements of the
//     task's stars (node i first, the others in a positively oriented order,
//     from the star word): cofactors, det, c_i, w = rho/120 (2 u_i + u_1 +
//     u_2 + u_3) + mu/(6 det) c_i, Codina's tau from h = det^(1/3) and the
//     velocity sum, the SUPG vector v = fs [(us . c_i) us + sum_n (u_n . c_i) u_n],
//     and the contributions (w + v) . c_k to its three entries; its record
//     goes to shared memory and its bit into those entries' masks.
//  3. Each off-diagonal entry lane adds, in element order, the records of its
//     masked elements: A + S, K += kv c_k x c_i + kd c_i x c_k, G's c_i sum and
//     det for the lumped mass.
//  4. A butterfly over the row's lanes gives every lane the row totals (FP64:
//     K and G summed in shared memory instead); the diagonal block is the
//     lumped mass times I minus the off-diagonal blocks' sum.
//  5. Every lane writes its own entry (the row's slice of each output array
//     is contiguous); the diagonal block's three compensated diagonal values
//     and the right-hand side are written by the row's lanes 0-5 (mixed32:
//     by the diagonal lane).
// Each element is evaluated once per row of its star (four times per tet).
// Long rows (more than 32 entries, or a star the row-gather encoder could
// not cover) are single-row tasks this kernel skips.
template <int P, bool DEBUG>
__global__ void __launch_bounds__(32 * STAR_WARPS, P == NSI_FP64 ? 1 : 6) stab_star_kernel(
    MeshView m, FieldView f, StabConst sc, const int4* __restrict__ tasks, int64_t ntasks,
    const uint16_t* __restrict__ star_word, void* Auu, void* Gv, void* rhs) {
  extern __shared__ __align__(16) unsigned char smem[];
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int CH = StarSmem<P>::CHUNK;
  const int lane = threadIdx.x & 31;
  const int64_t task = (int64_t)blockIdx.x * STAR_WARPS + (threadIdx.x >> 5);
  if (task >= ntasks) return;  // warp-uniform
  unsigned char* ws = smem + (threadIdx.x >> 5) * StarSmem<P>::bytes();
  T* er = reinterpret_cast<T*>(ws + StarSmem<P>::ent());
  T4<T>* el = reinterpret_cast<T4<T>*>(ws + StarSmem<P>::el());
  unsigned* mk = reinterpret_cast<unsigned*>(ws + StarSmem<P>::mask());  // [3 nodes][2 words][32 lanes]

  // the task's rows, CSR and star bounds and diagonal positions in one
  // 32-byte descriptor; long rows are left to the per-row kernel
  const int4 ta = tasks[2 * task], tb = tasks[2 * task + 1];
  if ((tb.w >> 24) & 1) return;  // warp-uniform
  const int nrow = (tb.w >> 16) & 3;  // 1 or 2
  const int64_t s0 = tb.x, s1 = tb.y, s2 = tb.z;
  const int nel = (int)(s2 - s0);
  // the first chunk's star words, loaded ahead of the rows' records
  unsigned wpre[2];
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) wpre[hf] = hf * 32 + lane < nel ? star_word[s0 + hf * 32 + lane] : 0u;
  const int width = nrow == 2 ? 16 : 32;
  const int seg = nrow == 2 ? lane >> 4 : 0;
  const int q = lane - seg * width;  // this lane's position in its row
  const int64_t i = (int64_t)ta.x + seg;
  const int32_t rs = seg ? ta.z : ta.y, len = (seg || nrow == 1 ? ta.w : ta.z) - rs;
  const int dp = seg ? (tb.w >> 8) & 255 : tb.w & 255;
  if (DEBUG && __any_sync(FULL, len > width || (len > 0 && dp >= len))) {  // warp-uniform
    if (lane == 0) atomicOr(m.err, ERR_STAR);
    return;
  }
  const bool has = q < len;
  const T kc = kc_of<T>(f), kmu = kmu_of<T>(f), kmass = kmass_of<T>(f);
  const StabK<T> sk = stab_k<T>(sc);
  const T kg = (T)(-1.0 / 24.0);

  // 1. entry records
  {
    const int j = has ? m.col_idx[rs + q] : 0;
    if (DEBUG && has && (j < 0 || j >= m.n)) atomicOr(m.err, ERR_BAD_INDEX);
    const int dl = seg * width + (len > 0 ? dp : 0);  // the diagonal's lane
    V3<T> d, u;
    if constexpr (P == NSI_FP64) {
      D4 x{0.0, 0.0, 0.0, 0.0}, v{0.0, 0.0, 0.0, 0.0};
      if (has && (!DEBUG || (j >= 0 && j < m.n))) {
        const D4* r = static_cast<const D4*>(m.rec) + 2 * (int64_t)j;
        x = r[0];
        v = r[1];
      }
      const double xi = __shfl_sync(FULL, x.x, dl), yi = __shfl_sync(FULL, x.y, dl), zi = __shfl_sync(FULL, x.z, dl);
      d = {x.x - xi, x.y - yi, x.z - zi};
      u = {v.x, v.y, v.z};
    } else {
      uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
      if (has && (!DEBUG || (j >= 0 && j < m.n))) {
        // the 32-byte record (32-byte aligned; written by the pack kernel, a
        // separate launch) in one 256-bit load instead of two 128-bit ones:
        // 0.944 against 0.954 ms mixed64, 0.733 against 0.755 mixed32
        const unsigned* r = static_cast<const unsigned*>(m.rec) + 8 * (int64_t)j;
        asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
            : "l"(r));
      }
      const V3<float> hj{__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z)};
      const V3<float> lj = record_lo(__uint_as_float(b.z), __uint_as_float(b.w));
      const V3<float> hi{__shfl_sync(FULL, hj.x, dl), __shfl_sync(FULL, hj.y, dl), __shfl_sync(FULL, hj.z, dl)};
      const V3<float> li{__shfl_sync(FULL, lj.x, dl), __shfl_sync(FULL, lj.y, dl), __shfl_sync(FULL, lj.z, dl)};
      d = add(sub(hj, hi), sub(lj, li));
      u = {__uint_as_float(a.w), __uint_as_float(b.x), __uint_as_float(b.y)};
    }
    er[0 * 32 + lane] = d.x;
    er[1 * 32 + lane] = d.y;
    er[2 * 32 + lane] = d.z;
    er[3 * 32 + lane] = u.x;
    er[4 * 32 + lane] = u.y;
    er[5 * 32 + lane] = u.z;
  }
  __syncwarp();

  // 2-3. elements in chunks of 64, then the entries' sums
  const int dp0 = __shfl_sync(FULL, dp, 0), dp1 = __shfl_sync(FULL, dp, 16);
  const int len0 = __shfl_sync(FULL, len, 0), len1 = __shfl_sync(FULL, len, 16);
  // an entry's sums (the few elements of its edge) in plain T; the row
  // totals below are compensated in mixed64
  T sA = T(0), sD = T(0);
  T K[9], G[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int c = 0; c < 9; ++c) K[c] = T(0);
  for (int c0 = 0; c0 < nel; c0 += CH) {
#pragma unroll
    for (int w = 0; w < 6; ++w) mk[w * 32 + lane] = 0u;
    __syncwarp();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int slot = half * 32 + lane;
      const int t = c0 + slot;
      if (t < nel) {
        const int es = (nrow == 2 && s0 + t >= s1) ? 1 : 0;  // the element's row
        const int eb = es * width;
        const int edp = es ? dp1 : dp0;
        const unsigned w = c0 == 0 ? wpre[half] : star_word[s0 + t];
        const int pa = w & 31, pb = (w >> 5) & 31, pc = (w >> 10) & 31;
        const int elen = es ? len1 : len0;
        if (DEBUG && (pa >= elen || pb >= elen || pc >= elen || elen > width)) {
          atomicOr(m.err, ERR_STAR);  // the element is left out
          continue;
        }
        auto rd = [&](int l, int c) { return V3<T>{er[c * 32 + l], er[(c + 1) * 32 + l], er[(c + 2) * 32 + l]}; };
        const V3<T> d1 = rd(eb + pa, 0), d2 = rd(eb + pb, 0), d3 = rd(eb + pc, 0);
        const V3<T> u1 = rd(eb + pa, 3), u2 = rd(eb + pb, 3), u3 = rd(eb + pc, 3), ui = rd(eb + edp, 3);
        const V3<T> c1 = cross(d2, d3), c2 = cross(d3, d1), c3 = cross(d1, d2);
        const T det = dot(d1, c1);
        const V3<T> ci{-(c1.x + c2.x + c3.x), -(c1.y + c2.y + c3.y), -(c1.z + c2.z + c3.z)};
        const T rdet = rcp_fast(det);
        const T kv = kmu * rdet;
        const V3<T> us = add(add(ui, u1), add(u2, u3));
        T h, sh;
        tau_lengths(det, dot(us, us), h, sh);
        const T fs = sk.ks * rcp_fast(h * fma_of(sk.krh, sh, sk.k4mu));
        const T kd = fma_of(sk.kr48 * sh, rdet, kv);
        const T as = fs * dot(us, ci), ai = fs * dot(ui, ci), a1 = fs * dot(u1, ci), a2 = fs * dot(u2, ci),
                a3 = fs * dot(u3, ci);
        // w + v: Galerkin convection and viscosity plus the SUPG vector
        V3<T> wv;
        wv.x = kc * (ui.x + us.x) + kv * ci.x + (as * us.x + ai * ui.x + a1 * u1.x + a2 * u2.x + a3 * u3.x);
        wv.y = kc * (ui.y + us.y) + kv * ci.y + (as * us.y + ai * ui.y + a1 * u1.y + a2 * u2.y + a3 * u3.y);
        wv.z = kc * (ui.z + us.z) + kv * ci.z + (as * us.z + ai * ui.z + a1 * u1.z + a2 * u2.z + a3 * u3.z);
        T4<T>* r = el + 5 * slot;
        r[0] = T4<T>{ci.x, ci.y, ci.z, kv};
        r[1] = T4<T>{c1.x, c1.y, c1.z, dot(wv, c1)};
        r[2] = T4<T>{c2.x, c2.y, c2.z, dot(wv, c2)};
        r[3] = T4<T>{c3.x, c3.y, c3.z, dot(wv, c3)};
        r[4] = T4<T>{kd, det, T(0), T(0)};
        const unsigned bit = 1u << lane;
        atomicOr(&mk[(0 * 2 + half) * 32 + eb + pa], bit);
        atomicOr(&mk[(1 * 2 + half) * 32 + eb + pb], bit);
        atomicOr(&mk[(2 * 2 + half) * 32 + eb + pc], bit);
      }
    }
    __syncwarp();
    if (has && q != dp) {
      const unsigned long long m1 = mk[2 * 32 + lane] | ((unsigned long long)mk[3 * 32 + lane] << 32);
      const unsigned long long m2 = mk[4 * 32 + lane] | ((unsigned long long)mk[5 * 32 + lane] << 32);
      unsigned long long bits = mk[0 * 32 + lane] | ((unsigned long long)mk[1 * 32 + lane] << 32) | m1 | m2;
      while (bits) {
        const int e = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        const int k = ((m1 >> e) & 1ull) ? 2 : ((m2 >> e) & 1ull) ? 3 : 1;
        const T4<T>* r = el + 5 * e;
        const T4<T> r0v = r[0], rk = r[k], r4 = r[4];
        sA += rk.w;
        sD += r4.y;
        const T kv = r0v.w, kd = r4.x;
        const T ri[3] = {r0v.x, r0v.y, r0v.z}, c[3] = {rk.x, rk.y, rk.z};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2)
            K[3 * a + b2] = fma_of(kv * c[a], ri[b2], fma_of(kd * ri[a], c[b2], K[3 * a + b2]));
        G[0] += ri[0];
        G[1] += ri[1];
        G[2] += ri[2];
      }
    }
    __syncwarp();
  }

  // 4. row totals (lanes without an off-diagonal entry hold zeros).  The
  // merge adds the error terms first (a commutative sum), so both lanes of a
  // butterfly pair, and in the end every lane of the row, hold bitwise the
  // same totals.
  auto merge_sym = [](Acc<P>& a, const Acc<P>& b) {
    if constexpr (P == NSI_MIXED_F32_ACC64) {
      a.lo += b.lo;
      a.add(b.hi);
    } else {
      a.v += b.v;
    }
  };
  Acc<P> tA, tD;
  tA.zero();
  tD.zero();
  tA.add(sA);
  tD.add(sD);
  T tK[9], tG[3];
#pragma unroll
  for (int c = 0; c < 9; ++c) tK[c] = K[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) tG[c] = G[c];
  for (int o = 1; o < width; o <<= 1) {
    Acc<P> xA, xD;
    if constexpr (P == NSI_MIXED_F32_ACC64) {
      xA.hi = __shfl_xor_sync(FULL, tA.hi, o);
      xA.lo = __shfl_xor_sync(FULL, tA.lo, o);
      xD.hi = __shfl_xor_sync(FULL, tD.hi, o);
      xD.lo = __shfl_xor_sync(FULL, tD.lo, o);
    } else {
      xA.v = __shfl_xor_sync(FULL, tA.v, o);
      xD.v = __shfl_xor_sync(FULL, tD.v, o);
    }
    merge_sym(tA, xA);
    merge_sym(tD, xD);
    if constexpr (P != NSI_FP64) {
#pragma unroll
      for (int c = 0; c < 9; ++c) tK[c] += __shfl_xor_sync(FULL, tK[c], o);
#pragma unroll
      for (int c = 0; c < 3; ++c) tG[c] += __shfl_xor_sync(FULL, tG[c], o);
    }
  }
  if constexpr (P == NSI_FP64) {
    // K and G totals in FP64 (a shuffled double is two shuffles): each lane's
    // values to shared memory (the element records' space, free now), the
    // row's lanes 0-11 each sum one value over the row's entries in lane
    // order, then every lane reads the totals
    T* red = reinterpret_cast<T*>(el);  // [32 lanes][13], then [2 rows][12] totals
    T* tot = red + 32 * 13;
#pragma unroll
    for (int c = 0; c < 9; ++c) red[lane * 13 + c] = K[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) red[lane * 13 + 9 + c] = G[c];
    __syncwarp();
    if (q < 12) {
      T sum = T(0);
      for (int r = 0; r < len; ++r) sum += red[(seg * width + r) * 13 + q];
      tot[seg * 12 + q] = sum;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 9; ++c) tK[c] = tot[seg * 12 + c];
#pragma unroll
    for (int c = 0; c < 3; ++c) tG[c] = tot[seg * 12 + 9 + c];
  }

  // 5. write-out: every lane its own entry.  mixed64 and FP64: the row's six
  // compensated values (the diagonal components of the diagonal block and
  // the right-hand side) by the row's lanes 0-5, one each, from the totals
  // every lane holds (the diagonal lane alone took them in turn: 2% of the
  // kernel in mixed64); mixed32, whose values are plain floats, keeps them on
  // the diagonal lane (the spread costs it 2%).
  Out* A = static_cast<Out*>(Auu);
  Out* Go = static_cast<Out*>(Gv);
  Out* Rh = static_cast<Out*>(rhs);
  if constexpr (P == NSI_MIXED_F32_ACC32) {
    if (has) {
      const int64_t g = (int64_t)rs + q;
      if (q == dp) {
        const Acc<P> mass = acc_scale<P>(acc_third<P>(tD), kmass);
#pragma unroll
        for (int c = 0; c < 9; ++c) A[c * m.nnz + g] = c % 4 == 0 ? mass.v - tA.v - tK[c] : -tK[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) Go[c * m.nnz + g] = tG[c] * (kg / T(3));
        const V3<T> un = load_vec<T>(f.un, i);
        Rh[i] = mass.v * un.x;
        Rh[m.n + i] = mass.v * un.y;
        Rh[2 * m.n + i] = mass.v * un.z;
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) A[c * m.nnz + g] = c % 4 == 0 ? sA + K[c] : K[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) Go[c * m.nnz + g] = G[c] * kg;
      }
    } else if (q == 0 && len == 0) {  // a node in no element: zero right-hand side
      Rh[i] = 0.0f;
      Rh[m.n + i] = 0.0f;
      Rh[2 * m.n + i] = 0.0f;
    }
  } else {
    if (has) {
      const int64_t g = (int64_t)rs + q;
      if (q == dp) {
#pragma unroll
        for (int c = 0; c < 9; ++c)
          if (c % 4 != 0) A[c * m.nnz + g] = (Out)(-tK[c]);
#pragma unroll
        for (int c = 0; c < 3; ++c) Go[c * m.nnz + g] = (Out)(tG[c] * (kg / T(3)));
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          A[c * m.nnz + g] = (Out)(c % 4 == 0 ? sA + K[c] : K[c]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) Go[c * m.nnz + g] = (Out)(G[c] * kg);
      }
    }
    if (len > 0 && q < 6) {  // (a row's lanes number 16 or 32)
      const Acc<P> mass = acc_scale<P>(acc_third<P>(tD), kmass);
      if (q < 3) {  // A(i,i)[c][c] = lumped mass - sum of the row's off-diagonal A - sum of K[c][c]
        Acc<P> x = mass;
        if constexpr (P == NSI_MIXED_F32_ACC64) {
          x.add(-tA.hi);
          x.lo -= tA.lo;
        } else {
          x.v = mass.v - tA.v;
        }
        x.add(-(q == 0 ? tK[0] : q == 1 ? tK[4] : tK[8]));
        store_acc(A + 4 * q * m.nnz + rs + dp, x);
      } else {  // rhs[k][i] = lumped mass * u^n_k
        const int k = q - 3;
        const T* un = static_cast<const T*>(k == 0 ? f.un[0] : k == 1 ? f.un[1] : f.un[2]);
        store_acc(Rh + k * m.n + i, acc_scale<P>(mass, __ldg(un + i)));
      }
    } else if (q == 0 && len == 0) {  // a node in no element: zero right-hand side
      Rh[i] = Out(0);
      Rh[m.n + i] = Out(0);
      Rh[2 * m.n + i] = Out(0);
    }
  }
}

// The stabilised block of listed rows (or of every row when `rows` is null),
// one thread per row in double whatever the handle's precision: the mixed
// modes' rows touching badly shaped elements, and whole meshes without an
// edge-fan map.  Each off-diagonal entry (i, j) sums the row's elements that
// contain j (node i first, the others in an even order so that det > 0), the
// diagonal block follows from the row totals as in the fan kernel.
template <int P>
__global__ void __launch_bounds__(64) stab_rows_kernel(MeshView m, FieldView f, StabConst sc, void* Auu, void* Gv,
                                                       void* rhs, const int32_t* rows, const int32_t* ptr,
                                                       const uint32_t* inc, int64_t count) {
  using Out = typename Prec<P>::Out;
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int64_t i = rows ? rows[r] : r;
  const int32_t rs = m.row_ptr[i], len = m.row_ptr[i + 1] - rs;
  const int32_t* cols = m.col_idx + rs;
  auto coord = [&](int64_t j) {
    if constexpr (P == NSI_FP64) {
      const D4 x = m.xyz64[j];
      return V3<double>{x.x, x.y, x.z};
    } else {
      const float4 h = m.xyz_hi[j], l = m.xyz_lo[j];
      return V3<double>{(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
    }
  };
  auto vel = [&](const void* const* comp, int64_t j) {
    if constexpr (P == NSI_FP64) return load_vec<double>(comp, j);
    else {
      const V3<float> w = load_vec<float>(comp, j);
      return V3<double>{w.x, w.y, w.z};
    }
  };
  const int EVEN[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
  const V3<double> xi = coord(i), ui = vel(f.u, i);
  const StabK<double> sk = stab_k<double>(sc);
  struct El {
    int v[3];
    V3<double> c[3], ci, u[3];
    double det;
  };
  auto element = [&](int32_t t) {
    El el;
    const int64_t e = inc[t] >> 2;
    const int a = (int)(inc[t] & 3u);
    const int4 v4 = m.lnods[e];
    const int v[4] = {v4.x, v4.y, v4.z, v4.w};
    V3<double> d[3];
    for (int b = 0; b < 3; ++b) {
      el.v[b] = v[EVEN[a][b]];
      d[b] = sub(coord(el.v[b]), xi);
      el.u[b] = vel(f.u, el.v[b]);
    }
    el.c[0] = cross(d[1], d[2]);
    el.c[1] = cross(d[2], d[0]);
    el.c[2] = cross(d[0], d[1]);
    el.det = dot(d[0], el.c[0]);
    el.ci = V3<double>{-(el.c[0].x + el.c[1].x + el.c[2].x), -(el.c[0].y + el.c[1].y + el.c[2].y),
                       -(el.c[0].z + el.c[1].z + el.c[2].z)};
    return el;
  };
  double detsum = 0.0;
  for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) detsum += element(t).det;
  Out* A = static_cast<Out*>(Auu) + rs;
  Out* G = static_cast<Out*>(Gv) + rs;
  double sa = 0.0, sK[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, sg[3] = {0.0, 0.0, 0.0};
  int dpos = -1;
  for (int q = 0; q < len; ++q) {
    const int32_t j = cols[q];
    if (j == i) {
      dpos = q;
      continue;
    }
    double a = 0.0, K[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, g[3] = {0.0, 0.0, 0.0};
    for (int32_t t = ptr[r]; t < ptr[r + 1]; ++t) {
      const int4 v4 = m.lnods[inc[t] >> 2];
      if (v4.x != j && v4.y != j && v4.z != j && v4.w != j) continue;
      const El el = element(t);
      const int b = el.v[0] == j ? 0 : el.v[1] == j ? 1 : 2;
      const double kv = f.kmu / el.det;
      const V3<double> us2{2.0 * ui.x + el.u[0].x + el.u[1].x + el.u[2].x,
                           2.0 * ui.y + el.u[0].y + el.u[1].y + el.u[2].y,
                           2.0 * ui.z + el.u[0].z + el.u[1].z + el.u[2].z};
      const V3<double> w{f.kc * us2.x + kv * el.ci.x, f.kc * us2.y + kv * el.ci.y, f.kc * us2.z + kv * el.ci.z};
      a += dot(w, el.c[b]);
      a += stab_terms<double>(el.ci, el.c[b], el.det, ui, el.u[0], el.u[1], el.u[2], sk, f.kmu, K);
      g[0] += el.ci.x;
      g[1] += el.ci.y;
      g[2] += el.ci.z;
    }
    sa += a;
    for (int c = 0; c < 9; ++c) {
      sK[c] += K[c];
      A[c * m.nnz + q] = (Out)((c % 4 == 0 ? a : 0.0) + K[c]);
    }
    for (int d = 0; d < 3; ++d) {
      G[d * m.nnz + q] = (Out)(-g[d] / 24.0);
      sg[d] += g[d];
    }
  }
  if (dpos >= 0) {
    const double dm = f.kmass * detsum - sa;
    for (int c = 0; c < 9; ++c) A[c * m.nnz + dpos] = (Out)((c % 4 == 0 ? dm : 0.0) - sK[c]);
    for (int d = 0; d < 3; ++d) G[d * m.nnz + dpos] = (Out)(-sg[d] / 72.0);
  }
  const V3<double> un = vel(f.un, i);
  Out* Rh = static_cast<Out*>(rhs);
  Rh[i] = (Out)(f.kmass * detsum * un.x);
  Rh[m.n + i] = (Out)(f.kmass * detsum * un.y);
  Rh[2 * m.n + i] = (Out)(f.kmass * detsum * un.z);
}

template <int P, bool DEBUG>
__global__ void __launch_bounds__(128) gather_kernel(MeshView m, FieldView f, OutView o, GatherSmem lay,
                                                     int64_t block0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gather_rows<P, DEBUG>(m, f, o, (block0 + blockIdx.x) * blockDim.x, smem_raw, lay);
}

// The row gather as a persistent grid (one CTA per resident block slot): a
// CTA's next block of rows loads its bounds and row scalars while the current
// block walks, and copies its column indices and walk steps (into nb1 and the
// walk region, free after the walk) while the current block writes out.
template <int P, bool DEBUG>
__global__ void __launch_bounds__(128) gather_persistent_kernel(MeshView m, FieldView f, OutView o, GatherSmem lay,
                                                                int64_t nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using T = typename Prec<P>::T;
  int64_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  const int R = blockDim.x;
  AccSmem<P> acc(smem_raw + lay.acc(), lay.N());
  Phase0<T> p = load_phase0<P>(m, f, blk * R);
  issue_phase0<DEBUG>(m, smem_raw, lay, p);
  while (true) {
    BlockRows<T> b;
    if (!stage_records<P, DEBUG>(m, smem_raw, lay, acc, p, b, kc_of<T>(f))) return;
    const int64_t nxt = blk + gridDim.x;
    const bool more = nxt < nblocks;  // block-uniform
    Phase0<T> pn = p;
    if (more) pn = load_phase0<P>(m, f, nxt * R);
    gather_compute<P, DEBUG>(m, f, o, smem_raw, lay, acc, b);
    if (more) issue_phase0<DEBUG>(m, smem_raw, lay, pn);
    gather_writeout<P>(m, o, smem_raw, lay, acc, b);
    if (!more) return;
    blk = nxt;
    p = pn;
  }
}

// ------------------------------------------------------ batched kernel ---
struct BatchItem {
  MeshView m;
  FieldView f;
  OutView o;
  int64_t block0;  // first global block of this mesh
};
struct BatchArgs {
  int32_t count;
  int64_t total_blocks;
  BatchItem item[NSI_MAX_BATCH];
};

// the item (mesh) of global block b: the last item with block0 <= b
__device__ __forceinline__ const BatchItem& batch_item(const BatchArgs& args, int64_t b) {
  int lo = 0, hi = args.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (args.item[mid].block0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return args.item[lo];
}

// the node records of every mesh of a batch in one launch: block b packs the
// nodes of the batch's row block b (the row gather's blocks of R rows)
template <int P>
__global__ void __launch_bounds__(128) batched_pack_kernel(const __grid_constant__ BatchArgs args) {
  const BatchItem& it = batch_item(args, blockIdx.x);
  const int64_t i = (blockIdx.x - it.block0) * (int64_t)blockDim.x + threadIdx.x;
  if (i < it.m.n) pack_node<P>(it.m, it.f, const_cast<void*>(it.m.rec), i);
}

template <int P>
__global__ void __launch_bounds__(128) batched_kernel(const __grid_constant__ BatchArgs args, GatherSmem lay) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (P == NSI_MIXED_F32_ACC64) {
    // as gather_persistent_kernel: the next block's phase 0 runs under the
    // current block's write-out (the next block may belong to another mesh)
    using T = typename Prec<P>::T;
    int64_t b = blockIdx.x;
    if (b >= args.total_blocks) return;
    const int R = blockDim.x;
    AccSmem<P> acc(smem_raw + lay.acc(), lay.N());
    const BatchItem* it = &batch_item(args, b);
    Phase0<T> p = load_phase0<P>(it->m, it->f, (b - it->block0) * R);
    issue_phase0<false>(it->m, smem_raw, lay, p);
    while (true) {
      BlockRows<T> rows;
      stage_records<P, false>(it->m, smem_raw, lay, acc, p, rows, kc_of<T>(it->f));
      const int64_t nxt = b + gridDim.x;
      const bool more = nxt < args.total_blocks;  // block-uniform
      const BatchItem* itn = more ? &batch_item(args, nxt) : it;
      Phase0<T> pn = p;
      if (more) pn = load_phase0<P>(itn->m, itn->f, (nxt - itn->block0) * R);
      gather_compute<P, false>(it->m, it->f, it->o, smem_raw, lay, acc, rows);
      if (more) issue_phase0<false>(itn->m, smem_raw, lay, pn);
      gather_writeout<P>(it->m, it->o, smem_raw, lay, acc, rows);
      if (!more) return;
      b = nxt;
      it = itn;
      p = pn;
    }
  } else {
    for (int64_t b = blockIdx.x; b < args.total_blocks; b += gridDim.x) {
      const BatchItem& it = batch_item(args, b);
      gather_rows<P, false>(it.m, it.f, it.o, (b - it.block0) * blockDim.x, smem_raw, lay);
      __syncthreads();  // the next block reuses the shared records
    }
  }
}

// many meshes, edge-fan variant: a persistent grid strides over the fan
// blocks of all meshes (item.block0 counts fan blocks here)
template <int P>
__global__ void __launch_bounds__(FAN_BLOCK) batched_fan_kernel(const __grid_constant__ BatchArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int64_t b = blockIdx.x; b < args.total_blocks; b += gridDim.x) {
    int lo = 0, hi = args.count - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (args.item[mid].block0 <= b) lo = mid;
      else hi = mid - 1;
    }
    const BatchItem& it = args.item[lo];
    fan_block<P, false>(it.m, it.f, it.o, b - it.block0, smem_raw);
    __syncthreads();  // the next block reuses the shared records
  }
}

// ----------------------------------------------------------- VJP kernel ---
// One element's adjoint terms in arithmetic C (edge vectors d1, d2, d3 from
// node 0; velocities u and adjoint weights w of the 4 nodes):
//   g[m] = sum_a w_a A_e[a][m] + rho/120 sum_k (W_k + w_{m,k}) Gu[k]
//   returned: 1/(6 det) sum_{a,k} w_{a,k} c_a . Gu[k]   (the grad_mu term)
// with W = sum_a w_a and Gu[k][l] = sum_b u_{b,k} c_b[l] = det du^k/dx_l.
template <typename C>
__device__ __forceinline__ C vjp_element(const V3<C>& d1, const V3<C>& d2, const V3<C>& d3, const V3<C> (&u)[4],
                                         const V3<C> (&w)[4], C kc, C kmu, C kmass, V3<C> (&g)[4]) {
  V3<C> c[4];
  c[1] = cross(d2, d3);
  c[2] = cross(d3, d1);
  c[3] = cross(d1, d2);
  const C det = dot(d1, c[1]);
  c[0] = {-(c[1].x + c[2].x + c[3].x), -(c[1].y + c[2].y + c[3].y), -(c[1].z + c[2].z + c[3].z)};
  const V3<C> S = add(add(u[0], u[1]), add(u[2], u[3]));
  const V3<C> Ws = add(add(w[0], w[1]), add(w[2], w[3]));
  const C kv = kmu * rcp(det);
  const C km = det * kmass;
  V3<C> Gu[3];
  const C uk[4][3] = {{u[0].x, u[0].y, u[0].z}, {u[1].x, u[1].y, u[1].z}, {u[2].x, u[2].y, u[2].z},
                      {u[3].x, u[3].y, u[3].z}};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Gu[k] = {C(0), C(0), C(0)};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      Gu[k].x += uk[b][k] * c[b].x;
      Gu[k].y += uk[b][k] * c[b].y;
      Gu[k].z += uk[b][k] * c[b].z;
    }
  }
#pragma unroll
  for (int mm = 0; mm < 4; ++mm) {
    V3<C> acc = {C(0), C(0), C(0)};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      C Aam = kc * dot(add(S, u[a]), c[mm]) + kv * dot(c[a], c[mm]);
      if (a == mm) Aam += km;
      acc.x += w[a].x * Aam;
      acc.y += w[a].y * Aam;
      acc.z += w[a].z * Aam;
    }
    const C wk[3] = {Ws.x + w[mm].x, Ws.y + w[mm].y, Ws.z + w[mm].z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc.x += kc * wk[k] * Gu[k].x;
      acc.y += kc * wk[k] * Gu[k].y;
      acc.z += kc * wk[k] * Gu[k].z;
    }
    g[mm] = acc;
  }
  C s = C(0);
#pragma unroll
  for (int a = 0; a < 4; ++a) s += w[a].x * dot(c[a], Gu[0]) + w[a].y * dot(c[a], Gu[1]) + w[a].z * dot(c[a], Gu[2]);
  return s * (C)(1.0 / 6.0) * rcp(det);
}

// true if element e is marked in the bit mask of badly shaped elements
__device__ __forceinline__ bool marked(const uint32_t* __restrict__ mask, int64_t e) {
  return mask && ((mask[e >> 5] >> (e & 31)) & 1u);
}

// the element's coordinates, velocities and weights in double (the handle's
// copy of the coordinates: double, or the float hi + lo pair)
template <int P>
__device__ __forceinline__ V3<double> coord64(const MeshView& m, int64_t j) {
  if constexpr (P == NSI_FP64) {
    const D4 x = m.xyz64[j];
    return V3<double>{x.x, x.y, x.z};
  } else {
    const float4 h = m.xyz_hi[j], l = m.xyz_lo[j];
    return V3<double>{(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
  }
}
template <typename T>
__device__ __forceinline__ V3<double> vec64(const void* const* comp, int64_t j) {
  const V3<T> v = load_vec<T>(comp, j);
  return V3<double>{(double)v.x, (double)v.y, (double)v.z};
}

// The adjoint, one element per thread, in the handle's arithmetic; the
// elements marked in `skip` (badly shaped, mixed modes) are left to
// vjp_exact_kernel.
template <int P>
__global__ void __launch_bounds__(256) vjp_kernel(MeshView m, FieldView f, const void* __restrict__ wv, void* gu,
                                                  double* gmu, const uint32_t* __restrict__ skip) {
  using T = typename Prec<P>::T;
  __shared__ T red[32];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T my_mu = T(0);
  if (e < m.E && !marked(skip, e)) {
    const int4 q = m.lnods[e];
    const int v[4] = {q.x, q.y, q.z, q.w};
    const T* W = static_cast<const T*>(wv);
    NodeX<P> X[4];
    V3<T> u[4], w[4], g[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      X[a].load(m, v[a]);
      u[a] = load_vec<T>(f.u, v[a]);
      w[a] = {W[v[a]], W[m.n + v[a]], W[2 * m.n + v[a]]};
    }
    my_mu = vjp_element<T>(X[1].minus(X[0]), X[2].minus(X[0]), X[3].minus(X[0]), u, w, kc_of<T>(f), kmu_of<T>(f),
                           kmass_of<T>(f), g);
    T* gp = static_cast<T*>(gu);
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
      atomicAdd(gp + v[mm], g[mm].x);
      atomicAdd(gp + m.n + v[mm], g[mm].y);
      atomicAdd(gp + 2 * m.n + v[mm], g[mm].z);
    }
  }
  // block reduction of the viscosity sensitivity
  for (int off = 16; off > 0; off >>= 1) my_mu += __shfl_down_sync(0xffffffffu, my_mu, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = my_mu;
  __syncthreads();
  if (threadIdx.x < 32) {
    T s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) {
      if constexpr (sizeof(T) == 4) atomicAdd(gmu, __longlong_as_double(f32_to_f64_bits(s)));
      else atomicAdd(gmu, (double)s);
    }
  }
}

// the badly shaped elements of the mixed modes in double (their determinant
// in float would carry about their shape ratio times the float rounding)
template <int P>
__global__ void __launch_bounds__(64) vjp_exact_kernel(MeshView m, FieldView f, const void* __restrict__ wv, void* gu,
                                                        double* gmu, const int32_t* __restrict__ list, int64_t count) {
  using T = typename Prec<P>::T;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = list[t];
  const int4 q = m.lnods[e];
  const int v[4] = {q.x, q.y, q.z, q.w};
  const void* wc[3] = {static_cast<const T*>(wv), static_cast<const T*>(wv) + m.n, static_cast<const T*>(wv) + 2 * m.n};
  V3<double> X[4], u[4], w[4], g[4];
  for (int a = 0; a < 4; ++a) {
    X[a] = coord64<P>(m, v[a]);
    u[a] = vec64<T>(f.u, v[a]);
    w[a] = vec64<T>(wc, v[a]);
  }
  const double mu = vjp_element<double>(sub(X[1], X[0]), sub(X[2], X[0]), sub(X[3], X[0]), u, w, f.kc, f.kmu, f.kmass, g);
  T* gp = static_cast<T*>(gu);
  for (int mm = 0; mm < 4; ++mm) {
    atomicAdd(gp + v[mm], (T)g[mm].x);
    atomicAdd(gp + m.n + v[mm], (T)g[mm].y);
    atomicAdd(gp + 2 * m.n + v[mm], (T)g[mm].z);
  }
  atomicAdd(gmu, mu);
}


// ----------------------------------------------------- residual kernel ---
// R[k][v_a] += sum_b A_e[a][b] u_b[k] - rho |T_e| / (4 dt) u^n_a[k]: the
// residual of the assembled system without forming A (element per thread).
template <typename C>
__device__ __forceinline__ void residual_element(const V3<C>& d1, const V3<C>& d2, const V3<C>& d3,
                                                 const V3<C> (&u)[4], const V3<C> (&un)[4], C kc, C kmu, C kmass,
                                                 V3<C> (&r)[4]) {
  V3<C> c[4];
  c[1] = cross(d2, d3);
  c[2] = cross(d3, d1);
  c[3] = cross(d1, d2);
  const C det = dot(d1, c[1]);
  c[0] = {-(c[1].x + c[2].x + c[3].x), -(c[1].y + c[2].y + c[3].y), -(c[1].z + c[2].z + c[3].z)};
  const V3<C> S = add(add(u[0], u[1]), add(u[2], u[3]));
  const C kv = kmu * rcp(det);
  const C km = det * kmass;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const V3<C> va = add(S, u[a]);
    V3<C> ra = {km * (u[a].x - un[a].x), km * (u[a].y - un[a].y), km * (u[a].z - un[a].z)};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const C Aab = kc * dot(va, c[b]) + kv * dot(c[a], c[b]);
      ra.x += Aab * u[b].x;
      ra.y += Aab * u[b].y;
      ra.z += Aab * u[b].z;
    }
    r[a] = ra;
  }
}

template <int P>
__global__ void __launch_bounds__(256) residual_kernel(MeshView m, FieldView f, void* rout,
                                                       const uint32_t* __restrict__ skip) {
  using T = typename Prec<P>::T;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E || marked(skip, e)) return;
  const int4 q = m.lnods[e];
  const int v[4] = {q.x, q.y, q.z, q.w};
  NodeX<P> X[4];
  V3<T> u[4], un[4], r[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a].load(m, v[a]);
    u[a] = load_vec<T>(f.u, v[a]);
    un[a] = load_vec<T>(f.un, v[a]);
  }
  residual_element<T>(X[1].minus(X[0]), X[2].minus(X[0]), X[3].minus(X[0]), u, un, kc_of<T>(f), kmu_of<T>(f),
                      kmass_of<T>(f), r);
  T* R = static_cast<T*>(rout);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    atomicAdd(R + v[a], r[a].x);
    atomicAdd(R + m.n + v[a], r[a].y);
    atomicAdd(R + 2 * m.n + v[a], r[a].z);
  }
}

template <int P>
__global__ void __launch_bounds__(64) residual_exact_kernel(MeshView m, FieldView f, void* rout,
                                                             const int32_t* __restrict__ list, int64_t count) {
  using T = typename Prec<P>::T;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = list[t];
  const int4 q = m.lnods[e];
  const int v[4] = {q.x, q.y, q.z, q.w};
  V3<double> X[4], u[4], un[4], r[4];
  for (int a = 0; a < 4; ++a) {
    X[a] = coord64<P>(m, v[a]);
    u[a] = vec64<T>(f.u, v[a]);
    un[a] = vec64<T>(f.un, v[a]);
  }
  residual_element<double>(sub(X[1], X[0]), sub(X[2], X[0]), sub(X[3], X[0]), u, un, f.kc, f.kmu, f.kmass, r);
  T* R = static_cast<T*>(rout);
  for (int a = 0; a < 4; ++a) {
    atomicAdd(R + v[a], (T)r[a].x);
    atomicAdd(R + m.n + v[a], (T)r[a].y);
    atomicAdd(R + 2 * m.n + v[a], (T)r[a].z);
  }
}

// --------------------------------------------- partition exchange ---
// The interface-row sum of a mesh split over ranks (disjoint element sets):
// values of chosen entries packed into an exchange buffer, and received
// values added into the owner's rows.
constexpr int XCH_MAX_COMP = 4;
struct CompPtrs {
  void* p[XCH_MAX_COMP];
};
// dst[k][c] = comp[c][idx[k]] (dst row-major [count][ncomp])
template <typename V>
__global__ void __launch_bounds__(256) gather_values_kernel(CompPtrs src, int ncomp, const int32_t* __restrict__ idx,
                                                            int64_t count, V* __restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int32_t i = idx[k];
  for (int c = 0; c < ncomp; ++c) dst[k * ncomp + c] = static_cast<const V*>(src.p[c])[i];
}
// comp[c][idx[k]] += src[k][c]; the positions of one call are distinct
template <typename V>
__global__ void __launch_bounds__(256) add_values_kernel(CompPtrs dst, int ncomp, const int32_t* __restrict__ idx,
                                                         int64_t count, const V* __restrict__ src) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int32_t i = idx[k];
  for (int c = 0; c < ncomp; ++c) static_cast<V*>(dst.p[c])[i] += src[k * ncomp + c];
}

// ----------------------------------------------------------- launchers ---
static nsi_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return NSI_OK;
}

template <int P>
static nsi_status zero_outputs(const NsiHandle* h, const OutView& o, cudaStream_t s) {
  using Out = typename Prec<P>::Out;
  NSI_CUDA(cudaMemsetAsync(o.A, 0, sizeof(Out) * h->nnz, s));
  NSI_CUDA(cudaMemsetAsync(o.G, 0, sizeof(Out) * 3 * h->nnz, s));
  NSI_CUDA(cudaMemsetAsync(o.rhs, 0, sizeof(Out) * 3 * h->n, s));
  return NSI_OK;
}

template <int P, bool DEBUG>
static nsi_status set_gather_smem() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(gather_kernel<P, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(gather_persistent_kernel<P, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(batched_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(gather smem)");
  return NSI_OK;
}

// after an assembly or time step in a mixed mode: the rows listed at create
// for badly shaped elements, recomputed in double (nothing if there are none)
template <int P>
static nsi_status fix_exact_rows(NsiHandle* h, const FieldView& f, int mode, void* A, void* G, void* rhs,
                                 void* dt_rho, void* mass_rho, double kmr, cudaStream_t s) {
  if constexpr (P == NSI_FP64) {
    return NSI_OK;
  } else {
    if (h->exact_rows == 0) return NSI_OK;
    const MeshView m = view_of(h);
    const int blk = 64;
    const int64_t grid = (h->exact_rows + blk - 1) / blk;
    if (mode == 0)
      exact_rows_kernel<P, 0><<<grid, blk, 0, s>>>(m, f, A, G, rhs, dt_rho, mass_rho, kmr, h->exact_list,
                                                  h->exact_ptr, h->exact_inc, h->exact_rows);
    else if (mode == 1)
      exact_rows_kernel<P, 1><<<grid, blk, 0, s>>>(m, f, A, G, rhs, dt_rho, mass_rho, kmr, h->exact_list,
                                                  h->exact_ptr, h->exact_inc, h->exact_rows);
    else
      exact_rows_kernel<P, 2><<<grid, blk, 0, s>>>(m, f, A, G, rhs, dt_rho, mass_rho, kmr, h->exact_list,
                                                  h->exact_ptr, h->exact_inc, h->exact_rows);
    return check_launch("exact_rows_kernel");
  }
}

// `rec` (nullptr: the handle's buffer) receives the row gather's per-call
// node records
// after any row-gather assembly or time step: the long rows (nothing if
// there are none)
template <int P>
static nsi_status fix_long_rows(NsiHandle* h, const FieldView& f, int mode, const void* A_static, void* A, void* G,
                                void* rhs, void* dt_rho, void* mass_rho, double kmr, cudaStream_t s) {
  if (h->long_rows == 0) return NSI_OK;
  const MeshView m = view_of(h);
  const int blk = 64;
  const int64_t grid = (h->long_rows + blk - 1) / blk;
  if (mode == 0)
    long_rows_kernel<P, 0><<<grid, blk, 0, s>>>(m, f, A_static, A, G, rhs, dt_rho, mass_rho, kmr, h->long_list,
                                               h->long_ptr, h->long_inc, h->long_rows);
  else if (mode == 1)
    long_rows_kernel<P, 1><<<grid, blk, 0, s>>>(m, f, A_static, A, G, rhs, dt_rho, mass_rho, kmr, h->long_list,
                                               h->long_ptr, h->long_inc, h->long_rows);
  else
    long_rows_kernel<P, 2><<<grid, blk, 0, s>>>(m, f, A_static, A, G, rhs, dt_rho, mass_rho, kmr, h->long_list,
                                               h->long_ptr, h->long_inc, h->long_rows);
  return check_launch("long_rows_kernel");
}

template <int P>
static nsi_status assemble_core_p(NsiHandle* h, const FieldView& f, const OutView& o, int mode, cudaStream_t s,
                                  void* rec = nullptr) {
  MeshView m = view_of(h);
  if (rec) m.rec = rec;
  const int blk = 256;
  if (mode == NSI_SCATTER_ATOMIC) {
    nsi_status st = zero_outputs<P>(h, o, s);
    if (st) return st;
    if (h->E == 0) return NSI_OK;
    const int64_t grid = (h->E + blk - 1) / blk;
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    // one atomic per value by default; the warp-aggregated variant issues 38%
    // fewer L2 reductions but about twice the instructions, slower on GB300
    // (100^3 cube: 2.19 against 2.60 ms mixed64, 1.81 against 1.89 mixed32,
    // 3.05 against 4.20 FP64); nsi_set_launch or the autotuner may select it
    if (h->atomic_agg) {
      if (h->debug) elem_kernel<P, true, true, true><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E, h->elem_pos);
      else elem_kernel<P, true, false, true><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E, h->elem_pos);
    } else {
      if (h->debug) elem_kernel<P, true, true><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E, h->elem_pos);
      else elem_kernel<P, true, false><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E, h->elem_pos);
    }
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    return check_launch("elem_kernel (atomic)");
  }
  if (mode == NSI_SCATTER_COLOR) {
    nsi_status st = zero_outputs<P>(h, o, s);
    if (st) return st;
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    for (int c = 0; c < h->n_colors; ++c) {
      const int64_t off = h->color_off[c], cnt = h->color_off[c + 1] - off;
      if (cnt == 0) continue;
      const int64_t grid = (cnt + blk - 1) / blk;
      if (h->debug) elem_kernel<P, false, true><<<grid, blk, 0, s>>>(m, f, o, h->color_elems + off, cnt, h->elem_pos);
      else elem_kernel<P, false, false><<<grid, blk, 0, s>>>(m, f, o, h->color_elems + off, cnt, h->elem_pos);
      nsi_status st2 = check_launch("elem_kernel (colour)");
      if (st2) return st2;
    }
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    return NSI_OK;
  }
  // row gather
  if (!h->gather_ok) return fail(NSI_ERR_UNSUPPORTED, "row-gather mode not available for this mesh");
  nsi_status st = h->debug ? set_gather_smem<P, true>() : set_gather_smem<P, false>();
  if (st) return st;
  pack_kernel<P><<<(h->n + 255) / 256, 256, 0, s>>>(m, f, const_cast<void*>(m.rec));
  if (h->use_fan) {
    const size_t fsm = FanSmem<P>::total(FAN_BLOCK);
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    if (h->debug) fan_kernel<P, true><<<h->fan_blocks, FAN_BLOCK, fsm, s>>>(m, f, o);
    else fan_kernel<P, false><<<h->fan_blocks, FAN_BLOCK, fsm, s>>>(m, f, o);
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    return check_launch("fan_kernel");
  }
  const int R = h->plan.rows_per_block;
  const GatherSmem lay = gather_smem(P, R, h->plan.w, h->plan.max_block_entries, h->plan.max_block_steps);
  const size_t smem = lay.total();
  if (h->persistent) {
    int per_sm = 0, sms = 0, dev = 0;
    NSI_CUDA(cudaGetDevice(&dev));
    NSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (h->debug)
      NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_persistent_kernel<P, true>, R, smem));
    else
      NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_persistent_kernel<P, false>, R, smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(h->plan.n_blocks, (int64_t)std::max(1, per_sm) * sms));
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    if (h->debug) gather_persistent_kernel<P, true><<<grid, R, smem, s>>>(m, f, o, lay, h->plan.n_blocks);
    else gather_persistent_kernel<P, false><<<grid, R, smem, s>>>(m, f, o, lay, h->plan.n_blocks);
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    return check_launch("gather_persistent_kernel");
  }
  if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
  if (h->debug) gather_kernel<P, true><<<h->plan.n_blocks, R, smem, s>>>(m, f, o, lay, 0);
  else gather_kernel<P, false><<<h->plan.n_blocks, R, smem, s>>>(m, f, o, lay, 0);
  if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
  return check_launch("gather_kernel");
}

template <int P>
static nsi_status assemble_p(NsiHandle* h, const FieldView& f, const OutView& o, int mode, cudaStream_t s) {
  nsi_status st = assemble_core_p<P>(h, f, o, mode, s);
  if (st) return st;
  st = fix_exact_rows<P>(h, f, 0, o.A, o.G, o.rhs, nullptr, nullptr, 0.0, s);
  if (st || mode != NSI_SCATTER_GATHER) return st;
  return fix_long_rows<P>(h, f, 0, nullptr, o.A, o.G, o.rhs, nullptr, nullptr, 0.0, s);
}

static nsi_status check_call(const NsiHandle* h, const NsiFields* f, const NsiOutputs* o) {
  if (!h || !f || !o) return fail(NSI_ERR_INVALID_ARG, "handle, fields or outputs is NULL");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if ((h->nnz > 0 && (!o->A_val || !o->G_val)) || !o->rhs)
    return fail(NSI_ERR_INVALID_ARG, "output pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  return NSI_OK;
}

static int resolve_mode(const NsiHandle* h, int mode) {
  if (mode == NSI_SCATTER_AUTO) mode = h->scatter;
  if (mode == NSI_SCATTER_AUTO) mode = h->gather_ok ? NSI_SCATTER_GATHER : NSI_SCATTER_ATOMIC;
  return mode;
}

static nsi_status assemble_dispatch(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, int mode,
                                    cudaStream_t s) {
  nsi_status st = check_call(h, f, o);
  if (st) return st;
  if (mode < NSI_SCATTER_AUTO || mode > NSI_SCATTER_GATHER) return fail(NSI_ERR_INVALID_ARG, "unknown scatter mode");
  mode = resolve_mode(h, mode);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != h->device) return fail(NSI_ERR_INVALID_ARG, "current device differs from the handle's device");
  const FieldView fv = fields_of(f);
  const OutView ov{o->A_val, o->G_val, o->rhs};
  switch (h->precision) {
    case NSI_FP64: return assemble_p<NSI_FP64>(h, fv, ov, mode, s);
    case NSI_MIXED_F32_ACC64: return assemble_p<NSI_MIXED_F32_ACC64>(h, fv, ov, mode, s);
    default: return assemble_p<NSI_MIXED_F32_ACC32>(h, fv, ov, mode, s);
  }
}

// the time-step kernels (convective step, nodal outputs): pack, then one
// step_kernel launch with the handle's rows per block
template <int P, bool NODAL, bool DEBUG>
static nsi_status set_step_smem() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(step_kernel<P, NODAL, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(step_persistent_kernel<P, NODAL, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
  });
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(step smem)");
  return NSI_OK;
}

template <int P, bool NODAL>
static nsi_status step_p(NsiHandle* h, const FieldView& f, const StepView& o, cudaStream_t s) {
  const MeshView m = view_of(h);
  nsi_status st = h->debug ? set_step_smem<P, NODAL, true>() : set_step_smem<P, NODAL, false>();
  if (st) return st;
  const int R = h->plan.rows_per_block;
  const GatherSmem lay = gather_smem(P, R, h->plan.w, h->plan.max_block_entries, h->plan.max_block_steps, true);
  const size_t smem = lay.total();
  if (smem > 200 * 1024) return fail(NSI_ERR_UNSUPPORTED, "the time-step layout needs more shared memory than a block has");
  pack_kernel<P><<<(h->n + 255) / 256, 256, 0, s>>>(m, f, h->rec);
  if constexpr (P == NSI_MIXED_F32_ACC32) {
    // the persistent grid measured faster for mixed32 only (0.235 against
    // 0.250 ms at the 100^3 cube; mixed64 0.321 against 0.291, FP64 2.38
    // against 2.17)
    int per_sm = 0, sms = 0, dev = 0;
    NSI_CUDA(cudaGetDevice(&dev));
    NSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (h->debug)
      NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_persistent_kernel<P, NODAL, true>, R, smem));
    else
      NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_persistent_kernel<P, NODAL, false>, R, smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(h->plan.n_blocks, (int64_t)std::max(1, per_sm) * sms));
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    if (h->debug) step_persistent_kernel<P, NODAL, true><<<grid, R, smem, s>>>(m, f, o, lay, h->plan.n_blocks);
    else step_persistent_kernel<P, NODAL, false><<<grid, R, smem, s>>>(m, f, o, lay, h->plan.n_blocks);
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    st = check_launch("step_persistent_kernel");
  } else {
    if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
    if (h->debug) step_kernel<P, NODAL, true><<<h->plan.n_blocks, R, smem, s>>>(m, f, o, lay);
    else step_kernel<P, NODAL, false><<<h->plan.n_blocks, R, smem, s>>>(m, f, o, lay);
    if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
    st = check_launch("step_kernel");
  }
  if (st) return st;
  st = fix_exact_rows<P>(h, f, NODAL ? 2 : 1, nullptr, nullptr, o.rhs, o.dt_rho, o.mass_rho, o.kmr, s);
  if (st) return st;
  return fix_long_rows<P>(h, f, NODAL ? 2 : 1, o.A_static, o.A, nullptr, o.rhs, o.dt_rho, o.mass_rho, o.kmr, s);
}

static nsi_status step_dispatch(NsiHandle* h, const NsiFields* f, const StepView& o, bool nodal, cudaStream_t s) {
  if (!h->gather_ok || h->n == 0)
    return h->n == 0 ? NSI_OK : fail(NSI_ERR_UNSUPPORTED, "the time-step kernels need the row-gather map");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != h->device) return fail(NSI_ERR_INVALID_ARG, "current device differs from the handle's device");
  const FieldView fv = fields_of(f);
  switch (h->precision) {
    case NSI_FP64:
      return nodal ? step_p<NSI_FP64, true>(h, fv, o, s) : step_p<NSI_FP64, false>(h, fv, o, s);
    case NSI_MIXED_F32_ACC64:
      return nodal ? step_p<NSI_MIXED_F32_ACC64, true>(h, fv, o, s) : step_p<NSI_MIXED_F32_ACC64, false>(h, fv, o, s);
    default:
      return nodal ? step_p<NSI_MIXED_F32_ACC32, true>(h, fv, o, s) : step_p<NSI_MIXED_F32_ACC32, false>(h, fv, o, s);
  }
}

template <int P>
static nsi_status batched_core_p(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os, int count,
                                 cudaStream_t s);

template <int P>
static nsi_status batched_p(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os, int count,
                            cudaStream_t s) {
  nsi_status st = batched_core_p<P>(hs, fs, os, count, s);
  for (int k = 0; k < count && !st; ++k) {
    st = fix_exact_rows<P>(hs[k], fields_of(&fs[k]), 0, os[k].A_val, os[k].G_val, os[k].rhs, nullptr, nullptr, 0.0,
                           s);
    if (!st)
      st = fix_long_rows<P>(hs[k], fields_of(&fs[k]), 0, nullptr, os[k].A_val, os[k].G_val, os[k].rhs, nullptr,
                            nullptr, 0.0, s);
  }
  return st;
}

template <int P>
static nsi_status batched_core_p(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os, int count,
                                 cudaStream_t s) {
  static BatchArgs args;  // host staging of the by-value kernel argument
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  args.count = count;
  bool all_fan = true;
  for (int k = 0; k < count; ++k) all_fan &= hs[k]->use_fan;
  if (all_fan) {
    int64_t fblocks = 0;
    for (int k = 0; k < count; ++k) {
      args.item[k].m = view_of(hs[k]);
      args.item[k].f = fields_of(&fs[k]);
      args.item[k].o = OutView{os[k].A_val, os[k].G_val, os[k].rhs};
      args.item[k].block0 = fblocks;
      fblocks += hs[k]->fan_blocks;
    }
    args.total_blocks = fblocks;
    if (fblocks == 0) return NSI_OK;
    for (int k = 0; k < count; ++k)
      pack_kernel<P><<<(hs[k]->n + 255) / 256, 256, 0, s>>>(args.item[k].m, args.item[k].f, hs[k]->rec);
    const size_t fsm = FanSmem<P>::total(FAN_BLOCK);
    int per_sm = 0, sms = 0, dev = 0;
    NSI_CUDA(cudaGetDevice(&dev));
    NSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_fan_kernel<P>, FAN_BLOCK, fsm));
    const int64_t grid = std::min<int64_t>(fblocks, (int64_t)std::max(1, per_sm) * sms);
    batched_fan_kernel<P><<<grid, FAN_BLOCK, fsm, s>>>(args);
    return check_launch("batched_fan_kernel");
  }
  // one block size for the whole batch: the largest one, no larger than any
  // mesh's own choice, that every mesh has planned (the per-block maxima of
  // the shared-memory layout are those of that size: blocks of different
  // sizes do not nest)
  int Rmin = 1 << 30, R = 0, max_entries = 0, max_steps = 0, max_row = 1;
  for (int k = 0; k < count; ++k) Rmin = std::min(Rmin, hs[k]->plan.rows_per_block);
  const GatherPlan* use[NSI_MAX_BATCH] = {};
  for (int cand : {128, 96, 64, 32}) {
    if (cand > Rmin) continue;
    bool all = true;
    for (int k = 0; k < count && all; ++k) {
      use[k] = nullptr;
      for (int j = 0; j < hs[k]->n_plans; ++j)
        if (hs[k]->plans[j].rows_per_block == cand) use[k] = &hs[k]->plans[j];
      all = use[k] != nullptr;
    }
    if (all) {
      R = cand;
      break;
    }
  }
  if (R == 0) return fail(NSI_ERR_UNSUPPORTED, "no block size is planned for every mesh of the batch");
  int64_t blocks = 0;
  for (int k = 0; k < count; ++k) {
    const NsiHandle* h = hs[k];
    max_entries = std::max(max_entries, use[k]->max_block_entries);
    max_steps = std::max(max_steps, use[k]->max_block_steps);
    max_row = std::max(max_row, use[k]->w);
    args.item[k].m = view_of(h);
    args.item[k].f = fields_of(&fs[k]);
    args.item[k].o = OutView{os[k].A_val, os[k].G_val, os[k].rhs};
    args.item[k].block0 = blocks;
    blocks += (h->n + R - 1) / R;
  }
  args.total_blocks = blocks;
  if (blocks == 0) return NSI_OK;
  batched_pack_kernel<P><<<blocks, R, 0, s>>>(args);
  nsi_status st = check_launch("batched_pack_kernel");
  if (st) return st;
  st = set_gather_smem<P, false>();
  if (st) return st;
  const GatherSmem lay = gather_smem(P, R, max_row, max_entries, max_steps);
  const size_t smem = lay.total();
  if (smem > 200 * 1024 || !lay.stage_fits())
    return fail(NSI_ERR_UNSUPPORTED, "batched meshes need more shared memory than a block has");
  int per_sm = 0, sms = 0, dev = 0;
  NSI_CUDA(cudaGetDevice(&dev));
  NSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<P>, R, smem));
  const int64_t grid = std::min<int64_t>(blocks, (int64_t)std::max(1, per_sm) * sms);
  batched_kernel<P><<<grid, R, smem, s>>>(args, lay);
  return check_launch("batched_kernel");
}

template <int P>
static nsi_status vjp_p(NsiHandle* h, const FieldView& f, const void* w, void* gu, double* gmu, cudaStream_t s) {
  using T = typename Prec<P>::T;
  NSI_CUDA(cudaMemsetAsync(gu, 0, sizeof(T) * 3 * h->n, s));
  NSI_CUDA(cudaMemsetAsync(gmu, 0, sizeof(double), s));
  if (h->E == 0) return NSI_OK;
  const int blk = 256;
  vjp_kernel<P><<<(h->E + blk - 1) / blk, blk, 0, s>>>(view_of(h), f, w, gu, gmu, h->bad_mask);
  nsi_status st = check_launch("vjp_kernel");
  if (st || h->n_bad == 0) return st;
  vjp_exact_kernel<P><<<(h->n_bad + 63) / 64, 64, 0, s>>>(view_of(h), f, w, gu, gmu, h->bad_list, h->n_bad);
  return check_launch("vjp_exact_kernel");
}


template <int P>
static nsi_status residual_p(NsiHandle* h, const FieldView& f, void* r, cudaStream_t s) {
  using T = typename Prec<P>::T;
  NSI_CUDA(cudaMemsetAsync(r, 0, sizeof(T) * 3 * h->n, s));
  if (h->E == 0) return NSI_OK;
  const int blk = 256;
  residual_kernel<P><<<(h->E + blk - 1) / blk, blk, 0, s>>>(view_of(h), f, r, h->bad_mask);
  nsi_status st = check_launch("residual_kernel");
  if (st || h->n_bad == 0) return st;
  residual_exact_kernel<P><<<(h->n_bad + 63) / 64, 64, 0, s>>>(view_of(h), f, r, h->bad_list, h->n_bad);
  return check_launch("residual_exact_kernel");
}

int gather_kernel_regs(int precision) {
  cudaFuncAttributes a{};
  cudaError_t e;
  if (precision == NSI_FP64) e = cudaFuncGetAttributes(&a, gather_kernel<NSI_FP64, false>);
  else if (precision == NSI_MIXED_F32_ACC64) e = cudaFuncGetAttributes(&a, gather_kernel<NSI_MIXED_F32_ACC64, false>);
  else e = cudaFuncGetAttributes(&a, gather_kernel<NSI_MIXED_F32_ACC32, false>);
  return e == cudaSuccess ? a.numRegs : 96;
}

// ------------------------------------------------ allocation-free variant ---
// Scratch of nsi_assemble_noalloc: room for the per-call node records of one
// mesh (32 bytes per node in the mixed modes, 64 in FP64).  It lives in the
// library's own device image, so every GPU that loads the library holds these
// 16 MiB until the process exits, and no call ever allocates it.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, and cached.
static nsi_status noalloc_scratch(int dev, void** out) {
  constexpr int MAX_DEV = 64;
  static std::mutex mu;
  static void* addr[MAX_DEV] = {};
  if (dev < 0 || dev >= MAX_DEV) return fail(NSI_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    NSI_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = p;
  }
  *out = addr[dev];
  return NSI_OK;
}

// the row gather of nsi_assemble (the same kernels and launch choice: star or
// edge-fan kernel, persistent grid, debug checks) with the node records in
// the static scratch, then the double-precision rows of badly shaped elements
template <int P>
static nsi_status assemble_noalloc_p(NsiHandle* h, const FieldView& f, const OutView& o, void* scratch,
                                     cudaStream_t s) {
  nsi_status st = assemble_core_p<P>(h, f, o, NSI_SCATTER_GATHER, s, scratch);
  if (st) return st;
  st = fix_exact_rows<P>(h, f, 0, o.A, o.G, o.rhs, nullptr, nullptr, 0.0, s);
  if (st) return st;
  return fix_long_rows<P>(h, f, 0, nullptr, o.A, o.G, o.rhs, nullptr, nullptr, 0.0, s);
}

}  // namespace nsi

using namespace nsi;

// Host-buffer call in the row-gather mode: the blocks of rows are assembled
// in chunks, and each finished chunk's slices of A, G and rhs go to the host
// on the handle's copy stream while the next chunk is assembled (the copies
// are the larger part of such a call).
template <int P>
static nsi_status host_chunked_p(NsiHandle* h, const NsiFields* fd, const NsiOutputs* od, const NsiOutputs* o,
                                 cudaStream_t s) {
  using Out = typename Prec<P>::Out;
  constexpr int C = (int)(sizeof(h->chunk_ev) / sizeof(h->chunk_ev[0]));
  if (!h->copy_stream) NSI_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : h->chunk_ev)
    if (!e) NSI_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  nsi_status st = h->debug ? set_gather_smem<P, true>() : set_gather_smem<P, false>();
  if (st) return st;
  const MeshView m = view_of(h);
  const FieldView fv = fields_of(fd);
  const OutView ov{od->A_val, od->G_val, od->rhs};
  const int R = h->plan.rows_per_block;
  const GatherSmem lay = gather_smem(P, R, h->plan.w, h->plan.max_block_entries, h->plan.max_block_steps);
  const size_t smem = lay.total();
  pack_kernel<P><<<(h->n + 255) / 256, 256, 0, s>>>(m, fv, h->rec);
  const int64_t nb = h->plan.n_blocks;
  const int chunks = (int)std::min<int64_t>(C, nb);
  const Out* dA = static_cast<const Out*>(od->A_val);
  const Out* dG = static_cast<const Out*>(od->G_val);
  const Out* dR = static_cast<const Out*>(od->rhs);
  Out* hA = static_cast<Out*>(o->A_val);
  Out* hG = static_cast<Out*>(o->G_val);
  Out* hR = static_cast<Out*>(o->rhs);
  // the link, not the kernel, bounds the call: a small first chunk starts the
  // copies early, later chunks grow (the kernel runs ahead of the copies)
  static_assert(C == 8, "chunk fractions are listed for 8 chunks");
  const double frac[C + 1] = {0.0, 1.0 / 64, 1.0 / 16, 3.0 / 16, 5.0 / 16, 0.5, 11.0 / 16, 27.0 / 32, 1.0};
  auto bound = [&](int c) {
    return chunks == C ? (int64_t)((double)nb * frac[c]) : nb * c / chunks;
  };
  for (int c = 0; c < chunks; ++c) {
    const int64_t b0 = bound(c), b1 = c + 1 == chunks ? nb : bound(c + 1);
    if (b1 <= b0) continue;
    if (h->debug) gather_kernel<P, true><<<b1 - b0, R, smem, s>>>(m, fv, ov, lay, b0);
    else gather_kernel<P, false><<<b1 - b0, R, smem, s>>>(m, fv, ov, lay, b0);
    st = check_launch("gather_kernel (host chunk)");
    if (st) return st;
    NSI_CUDA(cudaEventRecord(h->chunk_ev[c], s));
    NSI_CUDA(cudaStreamWaitEvent(h->copy_stream, h->chunk_ev[c], 0));
    const int64_t r0 = b0 * R, r1 = std::min<int64_t>(h->n, b1 * R);
    const int64_t e0 = h->row_ptr_host[r0], e1 = h->row_ptr_host[r1];
    const size_t eb = sizeof(Out) * (size_t)(e1 - e0), rb = sizeof(Out) * (size_t)(r1 - r0);
    // A's slice, then the three components of G and of rhs (equal slices at a
    // fixed pitch) as one 2D copy each
    NSI_CUDA(cudaMemcpyAsync(hA + e0, dA + e0, eb, cudaMemcpyDeviceToHost, h->copy_stream));
    const size_t gp = sizeof(Out) * (size_t)h->nnz, rp = sizeof(Out) * (size_t)h->n;
    NSI_CUDA(cudaMemcpy2DAsync(hG + e0, gp, dG + e0, gp, eb, 3, cudaMemcpyDeviceToHost, h->copy_stream));
    NSI_CUDA(cudaMemcpy2DAsync(hR + r0, rp, dR + r0, rp, rb, 3, cudaMemcpyDeviceToHost, h->copy_stream));
  }
  NSI_CUDA(cudaStreamSynchronize(h->copy_stream));
  NSI_CUDA(cudaStreamSynchronize(s));
  return NSI_OK;
}

template <int P, bool DEBUG>
static nsi_status set_star_smem() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(stab_star_kernel<P, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(StarSmem<P>::bytes() * STAR_WARPS));
  });
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(stabilised row kernel smem)");
  return NSI_OK;
}

// the stabilised velocity block: pack, the row kernel over every task, then
// the long rows and (mixed modes) the rows touching badly shaped elements by
// the per-row double kernel
template <int P>
static nsi_status stabilized_p(NsiHandle* h, const FieldView& f, const StabConst& sc, void* Auu, void* G, void* rhs,
                               cudaStream_t s) {
  if (h->n == 0) return NSI_OK;
  if (!h->gather_ok || !h->star_task)
    return fail(NSI_ERR_UNSUPPORTED, "the stabilised block needs the row maps (more than 2^31 node-element incidences)");
  nsi_status st = h->debug ? set_star_smem<P, true>() : set_star_smem<P, false>();
  if (st) return st;
  MeshView m = view_of(h);
  pack_kernel<P><<<(h->n + 255) / 256, 256, 0, s>>>(m, f, const_cast<void*>(m.rec));
  const size_t smem = StarSmem<P>::bytes() * STAR_WARPS;
  const int64_t grid = (h->n_star_tasks + STAR_WARPS - 1) / STAR_WARPS;
  if (h->ev_start) NSI_CUDA(cudaEventRecord(h->ev_start, s));
  if (h->debug)
    stab_star_kernel<P, true><<<grid, 32 * STAR_WARPS, smem, s>>>(m, f, sc, h->star_task, h->n_star_tasks,
                                                                   h->star_word, Auu, G, rhs);
  else
    stab_star_kernel<P, false><<<grid, 32 * STAR_WARPS, smem, s>>>(m, f, sc, h->star_task, h->n_star_tasks,
                                                                    h->star_word, Auu, G, rhs);
  if (h->ev_stop) NSI_CUDA(cudaEventRecord(h->ev_stop, s));
  st = check_launch("stab_star_kernel");
  if (st) return st;
  if (h->long_rows > 0) {
    stab_rows_kernel<P><<<(h->long_rows + 63) / 64, 64, 0, s>>>(m, f, sc, Auu, G, rhs, h->long_list, h->long_ptr,
                                                                 h->long_inc, h->long_rows);
    if ((st = check_launch("stab_rows_kernel (long rows)"))) return st;
  }
  if (P == NSI_FP64 || h->exact_rows == 0) return NSI_OK;
  stab_rows_kernel<P><<<(h->exact_rows + 63) / 64, 64, 0, s>>>(m, f, sc, Auu, G, rhs, h->exact_list, h->exact_ptr,
                                                                h->exact_inc, h->exact_rows);
  return check_launch("stab_rows_kernel (exact rows)");
}

extern "C" {

nsi_status nsi_assemble(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, void* stream) {
  return assemble_dispatch(h, f, o, NSI_SCATTER_AUTO, static_cast<cudaStream_t>(stream));
}

nsi_status nsi_assemble_mode(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, int32_t scatter, void* stream) {
  return assemble_dispatch(h, f, o, scatter, static_cast<cudaStream_t>(stream));
}

nsi_status nsi_assemble_batched(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os, int32_t count,
                                void* stream) {
  if (count < 0 || count > NSI_MAX_BATCH) return fail(NSI_ERR_INVALID_ARG, "count must be in [0, NSI_MAX_BATCH]");
  if (count == 0) return NSI_OK;
  if (!hs || !fs || !os) return fail(NSI_ERR_INVALID_ARG, "batch array is NULL");
  const int prec = hs[0] ? hs[0]->precision : -1;
  for (int k = 0; k < count; ++k) {
    nsi_status st = check_call(hs[k], &fs[k], &os[k]);
    if (st) return st;
    if (hs[k]->precision != prec) return fail(NSI_ERR_INVALID_ARG, "batched handles must share one precision");
    if (!hs[k]->gather_ok) return fail(NSI_ERR_UNSUPPORTED, "batched assembly needs the row-gather mode");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (prec) {
    case NSI_FP64: return batched_p<NSI_FP64>(hs, fs, os, count, s);
    case NSI_MIXED_F32_ACC64: return batched_p<NSI_MIXED_F32_ACC64>(hs, fs, os, count, s);
    default: return batched_p<NSI_MIXED_F32_ACC32>(hs, fs, os, count, s);
  }
}

nsi_status nsi_assemble_convective(NsiHandle* h, const NsiFields* f, const void* A_static, void* A_val, void* rhs,
                                   void* stream) {
  if (!h || !f || !rhs || (h->nnz > 0 && (!A_static || !A_val))) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  const StepView o{A_static, A_val, rhs, nullptr, nullptr, 0.0, 0.0f};
  return step_dispatch(h, f, o, false, static_cast<cudaStream_t>(stream));
}

nsi_status nsi_assemble_stabilized(NsiHandle* h, const NsiFields* f, void* Auu, void* G_val, void* rhs,
                                   void* stream) {
  if (!h || !f || !rhs || (h->nnz > 0 && (!Auu || !G_val))) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  if (!(f->mu > 0.0) || !std::isfinite(f->mu))
    return fail(NSI_ERR_INVALID_ARG, "mu must be finite and > 0 (tau1 of an element at rest is h^2 / (4 mu))");
  if (!(f->rho >= 0.0) || !std::isfinite(f->rho)) return fail(NSI_ERR_INVALID_ARG, "rho must be finite and >= 0");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != h->device) return fail(NSI_ERR_INVALID_ARG, "current device differs from the handle's device");
  const FieldView fv = fields_of(f);
  const StabConst sc = stab_const(f);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (h->precision) {
    case NSI_FP64: return stabilized_p<NSI_FP64>(h, fv, sc, Auu, G_val, rhs, s);
    case NSI_MIXED_F32_ACC64: return stabilized_p<NSI_MIXED_F32_ACC64>(h, fv, sc, Auu, G_val, rhs, s);
    default: return stabilized_p<NSI_MIXED_F32_ACC32>(h, fv, sc, Auu, G_val, rhs, s);
  }
}

nsi_status nsi_assemble_nodal(NsiHandle* h, const NsiFields* f, void* rhs, void* dt_rho, void* mass_rho, void* stream) {
  if (!h || !f || !rhs || !dt_rho || !mass_rho) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  const double kmr = f->rho / 24.0;
  const StepView o{nullptr, nullptr, rhs, dt_rho, mass_rho, kmr, (float)kmr};
  return step_dispatch(h, f, o, true, static_cast<cudaStream_t>(stream));
}

nsi_status nsi_assemble_vjp(NsiHandle* h, const NsiFields* f, const void* w, void* grad_u, double* grad_mu,
                            void* stream) {
  if (!h || !f || !w || !grad_u || !grad_mu) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  const FieldView fv = fields_of(f);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (h->precision) {
    case NSI_FP64: return vjp_p<NSI_FP64>(h, fv, w, grad_u, grad_mu, s);
    default: return vjp_p<NSI_MIXED_F32_ACC32>(h, fv, w, grad_u, grad_mu, s);
  }
}

nsi_status nsi_residual(NsiHandle* h, const NsiFields* f, void* r, void* stream) {
  if (!h || !f || !r) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!(f->dt > 0.0)) return fail(NSI_ERR_INVALID_ARG, "dt must be > 0");
  const FieldView fv = fields_of(f);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->precision == NSI_FP64) return residual_p<NSI_FP64>(h, fv, r, s);
  return residual_p<NSI_MIXED_F32_ACC32>(h, fv, r, s);
}

static nsi_status values_args(void* const* comp, int32_t ncomp, const int32_t* idx, int64_t count, const void* buf,
                              int32_t value_bytes, CompPtrs& cp) {
  if (count < 0) return fail(NSI_ERR_INVALID_ARG, "count < 0");
  if (ncomp < 1 || ncomp > XCH_MAX_COMP) return fail(NSI_ERR_INVALID_ARG, "ncomp must be in [1, 4]");
  if (value_bytes != 4 && value_bytes != 8) return fail(NSI_ERR_INVALID_ARG, "value_bytes must be 4 or 8");
  if (count > 0 && (!comp || !idx || !buf)) return fail(NSI_ERR_INVALID_ARG, "NULL argument");
  for (int c = 0; c < XCH_MAX_COMP; ++c) cp.p[c] = nullptr;
  for (int c = 0; c < ncomp && count > 0; ++c) {
    if (!comp[c]) return fail(NSI_ERR_INVALID_ARG, "NULL component pointer");
    cp.p[c] = comp[c];
  }
  return NSI_OK;
}

nsi_status nsi_gather_values(const void* const* src, int32_t ncomp, const int32_t* idx, int64_t count, void* dst,
                             int32_t value_bytes, void* stream) {
  CompPtrs cp;
  nsi_status st = values_args(const_cast<void* const*>(src), ncomp, idx, count, dst, value_bytes, cp);
  if (st || count == 0) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t grid = (count + 255) / 256;
  if (value_bytes == 8) gather_values_kernel<double><<<grid, 256, 0, s>>>(cp, ncomp, idx, count, static_cast<double*>(dst));
  else gather_values_kernel<float><<<grid, 256, 0, s>>>(cp, ncomp, idx, count, static_cast<float*>(dst));
  return check_launch("gather_values_kernel");
}

nsi_status nsi_add_values(void* const* dst, int32_t ncomp, const int32_t* idx, int64_t count, const void* src,
                          int32_t value_bytes, void* stream) {
  CompPtrs cp;
  nsi_status st = values_args(dst, ncomp, idx, count, src, value_bytes, cp);
  if (st || count == 0) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t grid = (count + 255) / 256;
  if (value_bytes == 8) add_values_kernel<double><<<grid, 256, 0, s>>>(cp, ncomp, idx, count, static_cast<const double*>(src));
  else add_values_kernel<float><<<grid, 256, 0, s>>>(cp, ncomp, idx, count, static_cast<const float*>(src));
  return check_launch("add_values_kernel");
}

nsi_status nsi_assemble_noalloc(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, void* stream) {
  nsi_status st = check_call(h, f, o);
  if (st) return st;
  if (!h->gather_ok) return fail(NSI_ERR_UNSUPPORTED, "the allocation-free call needs the row-gather mode");
  const size_t rec = h->precision == NSI_FP64 ? 64 : 32;
  if ((size_t)h->n * rec > NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "mesh too large for the allocation-free call: %lld nodes need %zu bytes of scratch, the static "
             "scratch holds %zu (%zu nodes at %zu bytes each)",
             (long long)h->n, (size_t)h->n * rec, NOALLOC_SCRATCH_BYTES, NOALLOC_SCRATCH_BYTES / rec, rec);
    return fail(NSI_ERR_UNSUPPORTED, buf);
  }
  int dev = 0;
  NSI_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return fail(NSI_ERR_INVALID_ARG, "current device differs from the handle's device");
  void* scratch = nullptr;
  st = noalloc_scratch(dev, &scratch);
  if (st) return st;
  const FieldView fv = fields_of(f);
  const OutView ov{o->A_val, o->G_val, o->rhs};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (h->precision) {
    case NSI_FP64: return assemble_noalloc_p<NSI_FP64>(h, fv, ov, scratch, s);
    case NSI_MIXED_F32_ACC64: return assemble_noalloc_p<NSI_MIXED_F32_ACC64>(h, fv, ov, scratch, s);
    default: return assemble_noalloc_p<NSI_MIXED_F32_ACC32>(h, fv, ov, scratch, s);
  }
}

nsi_status nsi_autotune(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, int32_t reps, void* stream,
                        int32_t* chosen_scatter, int32_t* chosen_rows) {
  nsi_status st = check_call(h, f, o);
  if (st) return st;
  if (reps < 1 || reps > 1000) return fail(NSI_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  NSI_CUDA(cudaEventCreate(&e0));
  NSI_CUDA(cudaEventCreate(&e1));
  struct Cand {
    int scatter, plan;  // plan: index into h->plans (star kernel), -2: edge-fan kernel,
                        // -3: warp-aggregated atomics, -1: n/a
  };
  std::vector<Cand> cands;
  if (h->fan_ok) cands.push_back({NSI_SCATTER_GATHER, -2});
  if (h->gather_ok)
    for (int k = 0; k < h->n_plans; ++k) cands.push_back({NSI_SCATTER_GATHER, k});
  cands.push_back({NSI_SCATTER_COLOR, -1});
  cands.push_back({NSI_SCATTER_ATOMIC, -1});
  cands.push_back({NSI_SCATTER_ATOMIC, -3});
  const GatherPlan saved = h->plan;
  const bool saved_fan = h->use_fan, saved_agg = h->atomic_agg;
  float best = 1e30f;
  Cand pick{h->scatter, saved_fan ? -2 : -1};
  cudaEvent_t ev0 = h->ev_start, ev1 = h->ev_stop;
  h->ev_start = h->ev_stop = nullptr;
  for (const Cand& c : cands) {
    h->use_fan = c.plan == -2;
    h->atomic_agg = c.plan == -3;
    if (c.plan >= 0) h->plan = h->plans[c.plan];
    st = assemble_dispatch(h, f, o, c.scatter, s);  // warm-up
    if (st) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && !st; ++r) st = assemble_dispatch(h, f, o, c.scatter, s);
    cudaEventRecord(e1, s);
    if (st) break;
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce != cudaSuccess) {
      st = cuda_fail(ce, "cudaEventSynchronize in autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  h->ev_start = ev0;
  h->ev_stop = ev1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->plan = pick.plan >= 0 ? h->plans[pick.plan] : saved;
  h->use_fan = pick.scatter == NSI_SCATTER_GATHER ? pick.plan == -2 : saved_fan;
  h->atomic_agg = pick.scatter == NSI_SCATTER_ATOMIC ? pick.plan == -3 : saved_agg;
  if (st) return st;
  h->scatter = pick.scatter;
  if (chosen_scatter) *chosen_scatter = pick.scatter;
  if (chosen_rows)
    *chosen_rows = pick.scatter == NSI_SCATTER_GATHER ? (h->use_fan ? -1 : h->plan.rows_per_block)
                   : pick.scatter == NSI_SCATTER_ATOMIC ? (h->atomic_agg ? 1 : 2)
                                                        : 0;
  return NSI_OK;
}

nsi_status nsi_assemble_host(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, void* stream) {
  nsi_status st = check_call(h, f, o);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t tsz = h->precision == NSI_FP64 ? 8 : 4;
  const size_t osz = h->precision == NSI_MIXED_F32_ACC32 ? 4 : 8;
  const bool sep_un = f->u_n[0] || f->u_n[1] || f->u_n[2];
  const size_t u_bytes = tsz * h->n * (sep_un ? 6 : 3);
  const size_t o_bytes = osz * (4 * h->nnz + 3 * h->n);
  const size_t need = ((u_bytes + 255) / 256) * 256 + o_bytes;
  if (h->stage_bytes < need) {
    cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    NSI_CUDA(cudaMalloc(&h->stage, need));
    h->stage_bytes = need;
  }
  char* base = static_cast<char*>(h->stage);
  NsiFields fd = *f;
  for (int k = 0; k < 3; ++k) {
    void* dst = base + k * tsz * h->n;
    NSI_CUDA(cudaMemcpyAsync(dst, f->u[k], tsz * h->n, cudaMemcpyHostToDevice, s));
    fd.u[k] = dst;
    fd.u_n[k] = nullptr;
  }
  if (sep_un) {
    for (int k = 0; k < 3; ++k) {
      void* dst = base + (3 + k) * tsz * h->n;
      const void* src = f->u_n[k] ? f->u_n[k] : f->u[k];
      NSI_CUDA(cudaMemcpyAsync(dst, src, tsz * h->n, cudaMemcpyHostToDevice, s));
      fd.u_n[k] = dst;
    }
  }
  char* ob = base + ((u_bytes + 255) / 256) * 256;
  NsiOutputs od{ob, ob + osz * h->nnz, ob + osz * 4 * h->nnz};
  if (resolve_mode(h, NSI_SCATTER_AUTO) == NSI_SCATTER_GATHER && !h->use_fan && h->n > 0 && h->exact_rows == 0 &&
      h->long_rows == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) return fail(NSI_ERR_INVALID_ARG, "current device differs from the handle's device");
    switch (h->precision) {
      case NSI_FP64: return host_chunked_p<NSI_FP64>(h, &fd, &od, o, s);
      case NSI_MIXED_F32_ACC64: return host_chunked_p<NSI_MIXED_F32_ACC64>(h, &fd, &od, o, s);
      default: return host_chunked_p<NSI_MIXED_F32_ACC32>(h, &fd, &od, o, s);
    }
  }
  st = assemble_dispatch(h, &fd, &od, NSI_SCATTER_AUTO, s);
  if (st) return st;
  NSI_CUDA(cudaMemcpyAsync(o->A_val, od.A_val, osz * h->nnz, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaMemcpyAsync(o->G_val, od.G_val, osz * 3 * h->nnz, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaMemcpyAsync(o->rhs, od.rhs, osz * 3 * h->n, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaStreamSynchronize(s));
  return NSI_OK;
}

}  // extern "C"
