// Device kernels and the per-call entry points of libnsi_assemble.
//
//   elem_kernel     one element per thread (calculate_transients ...
//                   perform_assembly_in_global_system of Listing 1 fused),
//                   scatter by global atomics or, colour by colour, by plain
//                   read-add-write (deterministic)
//   gather_kernel   one CSR row per thread: the row's owner visits every
//                   element around its node, accumulates the row privately
//                   and the block writes its contiguous slice of A, G and rhs
//                   once, coalesced (no atomics, no zeroing, deterministic)
//   batched_kernel  gather_kernel over many meshes in one persistent launch
//   vjp_kernel      adjoint of R(u, mu) = A(u) u - b, element per thread
//
// Formulas: see the element-arithmetic comment in nsi_internal.cuh.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "nsi_internal.cuh"

namespace nsi {

// ------------------------------------------------------------ views ------
struct MeshView {
  int64_t n, E, nnz;
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ col_idx;
  const int4* __restrict__ lnods;
  const int32_t* __restrict__ star_ptr;
  const uint16_t* __restrict__ star;
  const uint8_t* __restrict__ diag_pos;
  const D4* __restrict__ xyz64;
  const float4* __restrict__ xyz_hi;
  const float4* __restrict__ xyz_lo;
  unsigned* err;
};

struct FieldView {
  const void* u[3];
  const void* un[3];
  double rho, mu, dt;
};

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
  m.star_ptr = h->star_ptr;
  m.star = h->star;
  m.diag_pos = h->diag_pos;
  m.xyz64 = h->xyz64;
  m.xyz_hi = h->xyz_hi;
  m.xyz_lo = h->xyz_lo;
  m.err = h->err;
  return m;
}

static FieldView fields_of(const NsiFields* f) {
  FieldView v;
  for (int k = 0; k < 3; ++k) {
    v.u[k] = f->u[k];
    v.un[k] = f->u_n[k] ? f->u_n[k] : f->u[k];
  }
  v.rho = f->rho;
  v.mu = f->mu;
  v.dt = f->dt;
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
template <>
__device__ __forceinline__ void add_out<float, double>(double* p, float v, bool atomic) {
  double d = __longlong_as_double(f32_to_f64_bits(v));
  if (atomic) atomicAdd(p, d);  // the add itself happens in the L2 atomic unit
  else *p += d;
}

template <int P, bool ATOMIC, bool DEBUG>
__global__ void __launch_bounds__(256) elem_kernel(MeshView m, FieldView f, OutView o,
                                                   const int32_t* __restrict__ elems, int64_t count) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t e = elems ? (int64_t)elems[t] : t;
  const int4 q = m.lnods[e];
  const int v[4] = {q.x, q.y, q.z, q.w};
  if (DEBUG) {
    for (int a = 0; a < 4; ++a)
      if (v[a] < 0 || v[a] >= m.n) {
        atomicOr(m.err, ERR_BAD_INDEX);
        return;
      }
  }
  // gather (calculate_transients)
  NodeX<P> X[4];
  V3<T> u[4], un[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a].load(m, v[a]);
    u[a] = load_vec<T>(f.u, v[a]);
    un[a] = load_vec<T>(f.un, v[a]);
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
  const T kc = (T)(f.rho / 120.0);
  const T kv = (T)(f.mu / 6.0) * rcp(det);
  const T km = det * (T)(f.rho / (24.0 * f.dt));
  const T kg = (T)(-1.0 / 24.0);
  Out* A = static_cast<Out*>(o.A);
  Out* G = static_cast<Out*>(o.G);
  Out* R = static_cast<Out*>(o.rhs);
  // perform_assembly_in_global_system: locate the 4 columns in each row
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = v[a];
    const int rs = m.row_ptr[r], re = m.row_ptr[r + 1];
    int pos[4] = {-1, -1, -1, -1};
    for (int s = rs; s < re; ++s) {
      const int cidx = m.col_idx[s];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (cidx == v[b]) pos[b] = s;
    }
    const V3<T> va = add(S, u[a]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (DEBUG && pos[b] < 0) {
        atomicOr(m.err, ERR_NOT_IN_PATTERN);
        continue;
      }
      T Aab = kc * dot(va, c[b]) + kv * dot(c[a], c[b]);
      if (a == b) Aab += km;
      add_out<T, Out>(A + pos[b], Aab, ATOMIC);
      add_out<T, Out>(G + pos[b], kg * c[a].x, ATOMIC);
      add_out<T, Out>(G + m.nnz + pos[b], kg * c[a].y, ATOMIC);
      add_out<T, Out>(G + 2 * m.nnz + pos[b], kg * c[a].z, ATOMIC);
    }
    add_out<T, Out>(R + r, km * un[a].x, ATOMIC);
    add_out<T, Out>(R + m.n + r, km * un[a].y, ATOMIC);
    add_out<T, Out>(R + 2 * m.n + r, km * un[a].z, ATOMIC);
  }
}

// ---------------------------------------------------- row-gather kernel ---
// Accumulator of one output value: plain T, or a compensated float pair.
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

// shared-memory record of one CSR entry of the block: neighbour data (edge
// vector from the row's node and the neighbour's velocity) and the 4
// accumulators A, G_x, G_y, G_z of the entry
template <int P>
struct Entry {
  using T = typename Prec<P>::T;
  V3<T> d, u;
  Acc<P> a[4];
};

template <int P>
__host__ __device__ constexpr int entry_bytes() {
  return (int)sizeof(Entry<P>);
}

__device__ __forceinline__ void store_acc(double* p, const Acc<NSI_FP64>& a) { *p = a.v; }
__device__ __forceinline__ void store_acc(float* p, const Acc<NSI_MIXED_F32_ACC32>& a) { *p = a.v; }
__device__ __forceinline__ void store_acc(double* p, const Acc<NSI_MIXED_F32_ACC64>& a) {
  // renormalise the pair (Fast2Sum) so that |lo| <= ulp(hi)/2, then build the double
  float s = a.hi + a.lo;
  float lo = a.lo - (s - a.hi);
  *reinterpret_cast<long long*>(p) = pair_to_f64_bits(s, lo);
}

// one block of rows [r0, r0 + blockDim.x) of one mesh
template <int P, bool DEBUG>
__device__ __forceinline__ void gather_rows(const MeshView& m, const FieldView& f, const OutView& o, int64_t r0,
                                            Entry<P>* __restrict__ ent) {
  using T = typename Prec<P>::T;
  using Out = typename Prec<P>::Out;
  const int R = blockDim.x;
  const int64_t r_end = min(r0 + (int64_t)R, m.n);
  const int64_t i = r0 + threadIdx.x;
  const int32_t base = m.row_ptr[r0];
  const int32_t bend = m.row_ptr[r_end];
  const T kc = (T)(f.rho / 120.0);
  const T kmu = (T)(f.mu / 6.0);
  const T kmass = (T)(f.rho / (24.0 * f.dt));
  const T kg = (T)(-1.0 / 24.0);
  Out* A = static_cast<Out*>(o.A);
  Out* G = static_cast<Out*>(o.G);
  Out* Rh = static_cast<Out*>(o.rhs);

  if (i < r_end) {
    const int32_t rs = m.row_ptr[i], re = m.row_ptr[i + 1];
    const int len = re - rs;
    Entry<P>* row = ent + (rs - base);
    NodeX<P> xi;
    xi.load(m, i);
    const V3<T> ui = load_vec<T>(f.u, i);
    // stage the row's neighbours (calculate_transients for every element of the star)
    for (int q = 0; q < len; ++q) {
      const int j = m.col_idx[rs + q];
      if (DEBUG && (j < 0 || j >= m.n)) {
        atomicOr(m.err, ERR_BAD_INDEX);
        continue;
      }
      NodeX<P> xj;
      xj.load(m, j);
      row[q].d = xj.minus(xi);
      row[q].u = load_vec<T>(f.u, j);
#pragma unroll
      for (int c = 0; c < 4; ++c) row[q].a[c].zero();
    }
    // every element containing node i, with i as the local origin
    Acc<P> adiag, gdx, gdy, gdz, mass;
    adiag.zero();
    gdx.zero();
    gdy.zero();
    gdz.zero();
    mass.zero();
    const int32_t ss = m.star_ptr[i], se = m.star_ptr[i + 1];
    for (int32_t s = ss; s < se; ++s) {
      const unsigned w = m.star[s];
      const int p1 = w & 31, p2 = (w >> 5) & 31, p3 = (w >> 10) & 31;
      if (DEBUG && (p1 >= len || p2 >= len || p3 >= len)) {
        atomicOr(m.err, ERR_STAR);
        continue;
      }
      const V3<T> d1 = row[p1].d, d2 = row[p2].d, d3 = row[p3].d;
      const V3<T> u1 = row[p1].u, u2 = row[p2].u, u3 = row[p3].u;
      const V3<T> c1 = cross(d2, d3), c2 = cross(d3, d1), c3 = cross(d1, d2);
      const T det = dot(d1, c1);
      const V3<T> ci = {-(c1.x + c2.x + c3.x), -(c1.y + c2.y + c3.y), -(c1.z + c2.z + c3.z)};
      const V3<T> v = add(add(add(ui, ui), add(u1, u2)), u3);  // S + u_i
      const T kv = kmu * rcp(det);
      const V3<T> g = {kg * ci.x, kg * ci.y, kg * ci.z};
      row[p1].a[0].add(kc * dot(v, c1) + kv * dot(ci, c1));
      row[p2].a[0].add(kc * dot(v, c2) + kv * dot(ci, c2));
      row[p3].a[0].add(kc * dot(v, c3) + kv * dot(ci, c3));
      row[p1].a[1].add(g.x);
      row[p1].a[2].add(g.y);
      row[p1].a[3].add(g.z);
      row[p2].a[1].add(g.x);
      row[p2].a[2].add(g.y);
      row[p2].a[3].add(g.z);
      row[p3].a[1].add(g.x);
      row[p3].a[2].add(g.y);
      row[p3].a[3].add(g.z);
      const T km = kmass * det;
      adiag.add(kc * dot(v, ci) + kv * dot(ci, ci) + km);
      gdx.add(g.x);
      gdy.add(g.y);
      gdz.add(g.z);
      mass.add(km);
    }
    // diagonal entry of the row
    const int dp = m.diag_pos[i];
    if (len == 0) {
      // node in no element: empty row, zero right-hand side
    } else if (!DEBUG || dp < len) {
      row[dp].a[0] = adiag;
      row[dp].a[1] = gdx;
      row[dp].a[2] = gdy;
      row[dp].a[3] = gdz;
    } else {
      atomicOr(m.err, ERR_STAR);
    }
    // lumped RHS: (sum_e rho |T_e| / (4 dt)) u^n_i
    const V3<T> uni = load_vec<T>(f.un, i);
    const T unk[3] = {uni.x, uni.y, uni.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Acc<P> r;
      if constexpr (P == NSI_MIXED_F32_ACC64) {
        // (hi + lo) * u, keeping the product error (FMA-based TwoProd)
        float p = mass.hi * unk[k];
        float e = fmaf(mass.hi, unk[k], -p) + mass.lo * unk[k];
        r.hi = p;
        r.lo = e;
      } else {
        r.v = mass.v * unk[k];
      }
      store_acc(Rh + k * m.n + i, r);
    }
  }
  __syncthreads();
  // coalesced write of the block's contiguous slice of A and G
  for (int32_t t = threadIdx.x; t < bend - base; t += R) {
    const Entry<P>& en = ent[t];
    store_acc(A + base + t, en.a[0]);
    store_acc(G + base + t, en.a[1]);
    store_acc(G + m.nnz + base + t, en.a[2]);
    store_acc(G + 2 * m.nnz + base + t, en.a[3]);
  }
}

template <int P, bool DEBUG>
__global__ void __launch_bounds__(128) gather_kernel(MeshView m, FieldView f, OutView o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gather_rows<P, DEBUG>(m, f, o, (int64_t)blockIdx.x * blockDim.x, reinterpret_cast<Entry<P>*>(smem_raw));
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

template <int P>
__global__ void __launch_bounds__(128) batched_kernel(const __grid_constant__ BatchArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int64_t b = blockIdx.x; b < args.total_blocks; b += gridDim.x) {
    // mesh of global block b: last item with block0 <= b
    int lo = 0, hi = args.count - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (args.item[mid].block0 <= b) lo = mid;
      else hi = mid - 1;
    }
    const BatchItem& it = args.item[lo];
    gather_rows<P, false>(it.m, it.f, it.o, (b - it.block0) * blockDim.x, reinterpret_cast<Entry<P>*>(smem_raw));
    __syncthreads();  // the next block reuses the shared records
  }
}

// ----------------------------------------------------------- VJP kernel ---
// grad_u[l][v_m] += sum_a w_{a,l} A_e[a][m] + rho/120 sum_k (W_k + w_{m,k}) Gu[k][l]
// grad_mu       += 1/(6 det) sum_{a,k} w_{a,k} c_a . Gu[k]
// with W = sum_a w_a and Gu[k][l] = sum_b u_{b,k} c_b[l] = det du^k/dx_l.
template <int P>
__global__ void __launch_bounds__(256) vjp_kernel(MeshView m, FieldView f, const void* __restrict__ wv, void* gu,
                                                  double* gmu) {
  using T = typename Prec<P>::T;
  __shared__ T red[32];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T my_mu = T(0);
  if (e < m.E) {
    const int4 q = m.lnods[e];
    const int v[4] = {q.x, q.y, q.z, q.w};
    const T* W = static_cast<const T*>(wv);
    NodeX<P> X[4];
    V3<T> u[4], w[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      X[a].load(m, v[a]);
      u[a] = load_vec<T>(f.u, v[a]);
      w[a] = {W[v[a]], W[m.n + v[a]], W[2 * m.n + v[a]]};
    }
    const V3<T> d1 = X[1].minus(X[0]), d2 = X[2].minus(X[0]), d3 = X[3].minus(X[0]);
    V3<T> c[4];
    c[1] = cross(d2, d3);
    c[2] = cross(d3, d1);
    c[3] = cross(d1, d2);
    const T det = dot(d1, c[1]);
    c[0] = {-(c[1].x + c[2].x + c[3].x), -(c[1].y + c[2].y + c[3].y), -(c[1].z + c[2].z + c[3].z)};
    const V3<T> S = add(add(u[0], u[1]), add(u[2], u[3]));
    const V3<T> Ws = add(add(w[0], w[1]), add(w[2], w[3]));
    const T kc = (T)(f.rho / 120.0);
    const T kv = (T)(f.mu / 6.0) * rcp(det);
    const T km = det * (T)(f.rho / (24.0 * f.dt));
    // Gu[k] as vectors over l
    V3<T> Gu[3];
    const T uk[4][3] = {{u[0].x, u[0].y, u[0].z}, {u[1].x, u[1].y, u[1].z}, {u[2].x, u[2].y, u[2].z},
                        {u[3].x, u[3].y, u[3].z}};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Gu[k] = {T(0), T(0), T(0)};
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        Gu[k].x += uk[b][k] * c[b].x;
        Gu[k].y += uk[b][k] * c[b].y;
        Gu[k].z += uk[b][k] * c[b].z;
      }
    }
    T* g = static_cast<T*>(gu);
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
      V3<T> acc = {T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T Aam = kc * dot(add(S, u[a]), c[mm]) + kv * dot(c[a], c[mm]);
        if (a == mm) Aam += km;
        acc.x += w[a].x * Aam;
        acc.y += w[a].y * Aam;
        acc.z += w[a].z * Aam;
      }
      const T wk[3] = {Ws.x + w[mm].x, Ws.y + w[mm].y, Ws.z + w[mm].z};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc.x += kc * wk[k] * Gu[k].x;
        acc.y += kc * wk[k] * Gu[k].y;
        acc.z += kc * wk[k] * Gu[k].z;
      }
      atomicAdd(g + v[mm], acc.x);
      atomicAdd(g + m.n + v[mm], acc.y);
      atomicAdd(g + 2 * m.n + v[mm], acc.z);
    }
    T s = T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) s += w[a].x * dot(c[a], Gu[0]) + w[a].y * dot(c[a], Gu[1]) + w[a].z * dot(c[a], Gu[2]);
    my_mu = s * (T)(1.0 / 6.0) * rcp(det);
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


// ----------------------------------------------------- residual kernel ---
// R[k][v_a] += sum_b A_e[a][b] u_b[k] - rho |T_e| / (4 dt) u^n_a[k]: the
// residual of the assembled system without forming A (element per thread).
template <int P>
__global__ void __launch_bounds__(256) residual_kernel(MeshView m, FieldView f, void* rout) {
  using T = typename Prec<P>::T;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const int4 q = m.lnods[e];
  const int v[4] = {q.x, q.y, q.z, q.w};
  NodeX<P> X[4];
  V3<T> u[4], un[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    X[a].load(m, v[a]);
    u[a] = load_vec<T>(f.u, v[a]);
    un[a] = load_vec<T>(f.un, v[a]);
  }
  const V3<T> d1 = X[1].minus(X[0]), d2 = X[2].minus(X[0]), d3 = X[3].minus(X[0]);
  V3<T> c[4];
  c[1] = cross(d2, d3);
  c[2] = cross(d3, d1);
  c[3] = cross(d1, d2);
  const T det = dot(d1, c[1]);
  c[0] = {-(c[1].x + c[2].x + c[3].x), -(c[1].y + c[2].y + c[3].y), -(c[1].z + c[2].z + c[3].z)};
  const V3<T> S = add(add(u[0], u[1]), add(u[2], u[3]));
  const T kc = (T)(f.rho / 120.0);
  const T kv = (T)(f.mu / 6.0) * rcp(det);
  const T km = det * (T)(f.rho / (24.0 * f.dt));
  T* R = static_cast<T*>(rout);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const V3<T> va = add(S, u[a]);
    V3<T> r = {km * (u[a].x - un[a].x), km * (u[a].y - un[a].y), km * (u[a].z - un[a].z)};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const T Aab = kc * dot(va, c[b]) + kv * dot(c[a], c[b]);
      r.x += Aab * u[b].x;
      r.y += Aab * u[b].y;
      r.z += Aab * u[b].z;
    }
    atomicAdd(R + v[a], r.x);
    atomicAdd(R + m.n + v[a], r.y);
    atomicAdd(R + 2 * m.n + v[a], r.z);
  }
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
      err = cudaFuncSetAttribute(batched_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(gather smem)");
  return NSI_OK;
}

template <int P>
static nsi_status assemble_p(NsiHandle* h, const FieldView& f, const OutView& o, int mode, cudaStream_t s) {
  const MeshView m = view_of(h);
  const int blk = 256;
  if (mode == NSI_SCATTER_ATOMIC) {
    nsi_status st = zero_outputs<P>(h, o, s);
    if (st) return st;
    if (h->E == 0) return NSI_OK;
    const int64_t grid = (h->E + blk - 1) / blk;
    if (h->debug) elem_kernel<P, true, true><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E);
    else elem_kernel<P, true, false><<<grid, blk, 0, s>>>(m, f, o, nullptr, h->E);
    return check_launch("elem_kernel (atomic)");
  }
  if (mode == NSI_SCATTER_COLOR) {
    nsi_status st = zero_outputs<P>(h, o, s);
    if (st) return st;
    for (int c = 0; c < h->n_colors; ++c) {
      const int64_t off = h->color_off[c], cnt = h->color_off[c + 1] - off;
      if (cnt == 0) continue;
      const int64_t grid = (cnt + blk - 1) / blk;
      if (h->debug) elem_kernel<P, false, true><<<grid, blk, 0, s>>>(m, f, o, h->color_elems + off, cnt);
      else elem_kernel<P, false, false><<<grid, blk, 0, s>>>(m, f, o, h->color_elems + off, cnt);
      nsi_status st2 = check_launch("elem_kernel (colour)");
      if (st2) return st2;
    }
    return NSI_OK;
  }
  // row gather
  if (!h->gather_ok) return fail(NSI_ERR_UNSUPPORTED, "row-gather mode needs rows of at most 32 entries");
  nsi_status st = h->debug ? set_gather_smem<P, true>() : set_gather_smem<P, false>();
  if (st) return st;
  const size_t smem = (size_t)h->plan.max_block_entries * sizeof(Entry<P>);
  const int R = h->plan.rows_per_block;
  if (h->debug) gather_kernel<P, true><<<h->plan.n_blocks, R, smem, s>>>(m, f, o);
  else gather_kernel<P, false><<<h->plan.n_blocks, R, smem, s>>>(m, f, o);
  return check_launch("gather_kernel");
}

static nsi_status check_call(const NsiHandle* h, const NsiFields* f, const NsiOutputs* o) {
  if (!h || !f || !o) return fail(NSI_ERR_INVALID_ARG, "handle, fields or outputs is NULL");
  for (int k = 0; k < 3; ++k)
    if (!f->u[k]) return fail(NSI_ERR_INVALID_ARG, "velocity component pointer is NULL");
  if (!o->A_val || !o->G_val || !o->rhs) return fail(NSI_ERR_INVALID_ARG, "output pointer is NULL");
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

template <int P>
static nsi_status batched_p(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os, int count,
                            cudaStream_t s) {
  static BatchArgs args;  // host staging of the by-value kernel argument
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  args.count = count;
  int64_t blocks = 0;
  int R = 0, max_entries = 0;
  for (int k = 0; k < count; ++k) {
    const NsiHandle* h = hs[k];
    if (R == 0) R = h->plan.rows_per_block;
    if (h->plan.rows_per_block != R)
      return fail(NSI_ERR_UNSUPPORTED, "batched meshes must share one rows-per-block plan");
    max_entries = std::max(max_entries, h->plan.max_block_entries);
    args.item[k].m = view_of(h);
    args.item[k].f = fields_of(&fs[k]);
    args.item[k].o = OutView{os[k].A_val, os[k].G_val, os[k].rhs};
    args.item[k].block0 = blocks;
    blocks += h->plan.n_blocks;
  }
  args.total_blocks = blocks;
  if (blocks == 0) return NSI_OK;
  nsi_status st = set_gather_smem<P, false>();
  if (st) return st;
  const size_t smem = (size_t)max_entries * sizeof(Entry<P>);
  int per_sm = 0, sms = 0, dev = 0;
  NSI_CUDA(cudaGetDevice(&dev));
  NSI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<P>, R, smem));
  const int64_t grid = std::min<int64_t>(blocks, (int64_t)std::max(1, per_sm) * sms);
  batched_kernel<P><<<grid, R, smem, s>>>(args);
  return check_launch("batched_kernel");
}

template <int P>
static nsi_status vjp_p(NsiHandle* h, const FieldView& f, const void* w, void* gu, double* gmu, cudaStream_t s) {
  using T = typename Prec<P>::T;
  NSI_CUDA(cudaMemsetAsync(gu, 0, sizeof(T) * 3 * h->n, s));
  NSI_CUDA(cudaMemsetAsync(gmu, 0, sizeof(double), s));
  if (h->E == 0) return NSI_OK;
  const int blk = 256;
  vjp_kernel<P><<<(h->E + blk - 1) / blk, blk, 0, s>>>(view_of(h), f, w, gu, gmu);
  return check_launch("vjp_kernel");
}


template <int P>
static nsi_status residual_p(NsiHandle* h, const FieldView& f, void* r, cudaStream_t s) {
  using T = typename Prec<P>::T;
  NSI_CUDA(cudaMemsetAsync(r, 0, sizeof(T) * 3 * h->n, s));
  if (h->E == 0) return NSI_OK;
  const int blk = 256;
  residual_kernel<P><<<(h->E + blk - 1) / blk, blk, 0, s>>>(view_of(h), f, r);
  return check_launch("residual_kernel");
}

}  // namespace nsi

using namespace nsi;

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
  st = assemble_dispatch(h, &fd, &od, NSI_SCATTER_AUTO, s);
  if (st) return st;
  NSI_CUDA(cudaMemcpyAsync(o->A_val, od.A_val, osz * h->nnz, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaMemcpyAsync(o->G_val, od.G_val, osz * 3 * h->nnz, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaMemcpyAsync(o->rhs, od.rhs, osz * 3 * h->n, cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaStreamSynchronize(s));
  return NSI_OK;
}

}  // extern "C"
