// Mat-vec of Eqs. 5-6 (and its transpose) visiting every unordered pair once.
//
// The four kernels of a pair share r, e^{-kappa r}, t and w; only the dot
// products with the normals and the sign of d differ between the two
// directions.  Each work item is one tile of T targets of a system (row I)
// against a range of sources at or after the tile's first element; every pair
// (i, j) with j > i is evaluated once and applied both ways:
//   target i gathers source j      -> register accumulators (i side)
//   target j gathers source i      -> summed over the CTA's T targets (j side)
// In the tile's own diagonal block the pairs with j <= i are masked (1/r = 0).
// The j side of a source is summed over a warp by accumulators that rotate
// through the lanes, and over the warps in a fixed order, so results are
// bitwise reproducible.
//
// Row I of a system has n - I T sources, so rows shrink down the system.
// Rows I and nT - 1 - I are folded together (about n + T sources between
// them) and the folded rows are cut into pieces of equal length; a piece is
// one work item and covers one or two segments (tile, source range).  All
// items thus carry the same work, and their number is chosen to fill whole
// waves of resident CTAs.
//
// Partial sums (per system, T = targets per tile, nT tiles):
//   i side: one block of 2 x T values per segment (a row's segments are
//           numbered consecutively, in source order);
//   j side: for row I, 2 x (n - I T) values (every element j >= I T).
// The reduction adds, for element e of tile E, the i-side blocks of row E and
// the j-side values of rows 0..E, in that fixed order, in FP64.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <type_traits>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr double kInv4PiS = 1.0 / (4.0 * kPi);

template <typename T>
struct SymV4;
template <>
struct SymV4<float> {
  using type = float4;
};
template <>
struct SymV4<double> {
  using type = double4_32a;
};

// ------------------------------------------------------------------ policies
// Record of an element (both roles): position, a, normal, alpha, where
// (a, alpha) = (ds psi, ds phi) for A u and (wphi, wpsi) for A^T w.

// LAPLACE: the kappa = 0 form of sym_pair (pair.cuh); otherwise the records
// are in kappa-scaled units (SCALED).
template <typename T, bool TRANS, bool LAPLACE>
struct SymPolicy {
  using V4 = typename SymV4<T>::type;
  using PT = T;  // partial sums are stored in this type
  static constexpr bool SCALED = !LAPLACE;
  static constexpr int RW = 2;  // (x, a), (n, alpha)
  static constexpr int UNROLL = sizeof(T) == 4 ? 4 : 1;  // sources in flight per thread
  struct Elem {
    T x[3], a, n[3], al;
  };
  struct Acc {
    T p, q;
  };
  struct Args {
    PairConst<T> c;
  };
  __device__ static void prologue(const Args&) {}
  __device__ static void load(const V4* r, Elem& e) { unpack(r[0], r[1], e); }
  // record q of a chunk staged as planes (vector r of record q at sh[r * CH + q])
  template <int CH>
  __device__ static void load_plane(const V4* sh, int q, Elem& e) { unpack(sh[q], sh[CH + q], e); }
  __device__ static void unpack(const V4& A, const V4& B, Elem& e) {
    e.x[0] = A.x, e.x[1] = A.y, e.x[2] = A.z, e.a = A.w;
    e.n[0] = B.x, e.n[1] = B.y, e.n[2] = B.z, e.al = B.w;
  }
  __device__ static void zero(Acc& v) { v.p = T(0), v.q = T(0); }
  // i-side of target t and j-side of source sj for the pair d = x_t - x_sj
  template <bool MASK>
  __device__ static void pair(const Args& g, const Elem& t, const Elem& sj, bool masked, Acc& ti, Acc& tj) {
    sym_pair<MASK, TRANS, LAPLACE>(t.x[0] - sj.x[0], t.x[1] - sj.x[1], t.x[2] - sj.x[2], t.n, t.a, t.al, sj.n, sj.a, sj.al,
                          masked, g.c, ti.p, ti.q, tj.p, tj.q);
  }
  __device__ static void renorm(Acc&) {}
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T shfl_from(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  // a source slot q past the end of a chunk: far away, no field, no normal (adds exact zeros)
  template <int CH>
  __device__ static void pad(V4* sh, int q) {
    V4 z;
    z.x = T(1e4), z.y = T(1e4), z.z = T(1e4), z.w = T(0);
    sh[q] = z;
    z.x = z.y = z.z = T(0);
    sh[CH + q] = z;
  }
  __device__ static PT out(T v) { return v; }
};

__device__ df* sym_exp_table() {
  __shared__ __align__(16) df tab[kExpTab];
  return tab;
}

// df64 record, 4 float4: (x.hi, a.hi), (x.lo, a.lo), (n.hi, alpha.hi), (n.lo, alpha.lo);
// SCALED: positions and alpha in kappa-scaled units (df_sym_pair)
template <bool TRANS, bool SCALED_>
struct SymDFPolicy {
  using V4 = float4;
  using PT = double;
  static constexpr bool SCALED = SCALED_;
  static constexpr int RW = 4;
  static constexpr int UNROLL = 1;
  struct Elem {
    df x[3], a, n[3], al;
  };
  struct Acc {
    df p, q;
  };
  struct Args {
    DFConst c;
  };
  __device__ static void prologue(const Args& g) { df_load_exp_table(sym_exp_table(), g.c); }
  __device__ static void load(const float4* r, Elem& e) { unpack(r[0], r[1], r[2], r[3], e); }
  template <int CH>
  __device__ static void load_plane(const float4* sh, int q, Elem& e) {
    unpack(sh[q], sh[CH + q], sh[2 * CH + q], sh[3 * CH + q], e);
  }
  __device__ static void unpack(const float4& A, const float4& B, const float4& C, const float4& D, Elem& e) {
    e.x[0] = df{A.x, B.x}, e.x[1] = df{A.y, B.y}, e.x[2] = df{A.z, B.z}, e.a = df{A.w, B.w};
    e.n[0] = df{C.x, D.x}, e.n[1] = df{C.y, D.y}, e.n[2] = df{C.z, D.z}, e.al = df{C.w, D.w};
  }
  __device__ static void zero(Acc& v) { v.p = df{0.f, 0.f}, v.q = df{0.f, 0.f}; }
  template <bool MASK>
  __device__ static void pair(const Args& g, const Elem& t, const Elem& sj, bool masked, Acc& ti, Acc& tj) {
    const df d[3] = {df_sub(t.x[0], sj.x[0]), df_sub(t.x[1], sj.x[1]), df_sub(t.x[2], sj.x[2])};
    df_sym_pair<MASK, TRANS, SCALED>(d, t.n, t.a, t.al, sj.n, sj.a, sj.al, masked, g.c, sym_exp_table(), ti.p, ti.q,
                                     tj.p, tj.q);
  }
  // the accumulators are updated lazily (df_mac): bring them back to normal form
  __device__ static void renorm(Acc& v) {
    v.p = two_sum(v.p.hi, v.p.lo);
    v.q = two_sum(v.q.hi, v.q.lo);
  }
  __device__ static df add(df a, df b) { return df_add(a, b); }
  __device__ static df shfl_from(df v, int src) {
    return df{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
  }
  template <int CH>
  __device__ static void pad(float4* sh, int q) {
    sh[q] = make_float4(1e4f, 1e4f, 1e4f, 0.f);
    sh[CH + q] = sh[2 * CH + q] = sh[3 * CH + q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ static PT out(df v) { return df_to_double(v); }
};

// ------------------------------------------------------------------ kernel
// One shared-memory chunk of cnt sources (starting at j0) against the
// thread's TPT targets.  MASK: the chunk overlaps the tile's own targets, and
// pairs with j <= i are masked.  The j side rotates through the warp: the
// chunk is taken in blocks of 32 sources (the slots past cnt padded with
// records that add exact zeros); at step k of a block, lane l evaluates
// source (l + k) mod 32 against its targets, then takes over the accumulator
// of the next source from lane l + 1.  After 32 steps lane l holds the
// complete j-side sum of source (l + 31) mod 32 over the warp's targets,
// accumulated in a fixed order; it leaves it in jred[warp][source].
template <class P, int TPT, int CH, bool MASK>
__device__ __forceinline__ void sym_chunk(const typename P::Args& g, const typename P::Elem* tg, const int* idx,
                                              typename P::Acc* acc, const typename P::V4* sh, int cnt, int j0,
                                              typename P::Acc (*jred)[CH]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int next = (lane + 1) & 31;
  for (int r0 = 0; r0 < cnt; r0 += 32) {
    typename P::Acc tj;
    P::zero(tj);
#pragma unroll P::UNROLL
    for (int k = 0; k < 32; ++k) {
      const int jj = r0 + ((lane + k) & 31);
      typename P::Elem sj;
      P::template load_plane<CH>(sh, jj, sj);
#pragma unroll
      for (int t = 0; t < TPT; ++t) P::template pair<MASK>(g, tg[t], sj, MASK && j0 + jj <= idx[t], acc[t], tj);
      if (k < 31) {
        tj.p = P::shfl_from(tj.p, next);
        tj.q = P::shfl_from(tj.q, next);
      }
    }
    P::renorm(tj);
    const int mine = r0 + ((lane + 31) & 31);
    if (mine < cnt) jred[warp][mine] = tj;
  }
}

// Item (three int4): {rec_off, n, sys, jbase}, then two segments
// {t0, s0, s1, ioff} (s0 == s1: empty): targets t0 + [0, T) of a system with n
// elements whose records start at rec_off, against sources [s0, s1) (s0 >=
// t0); i-side partials at part[ioff + c T + i - t0], j-side at part[jrow +
// c (n - t0) + j - t0] with jrow the start of row t0 / T after jbase.
template <class P, int NT, int TPT, int CH, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_sym(typename P::Args g, const int4* __restrict__ items,
                                            const typename P::V4* __restrict__ rec, typename P::PT* __restrict__ part,
                                            const int* __restrict__ skip, int skip_stride) {
  using V4 = typename P::V4;
  using Acc = typename P::Acc;
  constexpr int NW = NT / 32, T = NT * TPT;
  __shared__ V4 sh[CH * P::RW];
  __shared__ Acc jred[NW][CH];
  chain_wait();  // the records of the pack kernel (no early release: this kernel is long)
  const int4 H = items[3 * blockIdx.x];
  const int rec_off = H.x, n = H.y, sys = H.z, jbase = H.w;
  if (skip != nullptr && skip[(size_t)sys * skip_stride] != 0) return;
  P::prologue(g);  // per-CTA shared tables (made visible by the first barrier below)
  for (int seg = 0; seg < 2; ++seg) {
    const int4 S = items[3 * blockIdx.x + 1 + seg];
    const int t0 = S.x, s0 = S.y, s1 = S.z, ioff = S.w;
    if (s0 >= s1) continue;
    const int I = t0 / T;
    const int64_t jrow = jbase + 2 * ((int64_t)I * n - (int64_t)T * I * (I - 1) / 2);
    const int len = n - t0;  // j-side row length
    typename P::Elem tg[TPT];
    Acc acc[TPT];
    int idx[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
      idx[k] = t0 + k * NT + threadIdx.x;
      P::load(rec + (size_t)(rec_off + min(idx[k], n - 1)) * P::RW, tg[k]);
      P::zero(acc[k]);
    }
    for (int j0 = s0; j0 < s1; j0 += CH) {
      const int cnt = min(CH, s1 - j0);
      __syncthreads();
      // stage the chunk as planes: vector r of record q at sh[r * CH + q] (the
      // lanes of a warp read consecutive records: no bank conflicts)
      const V4* src = rec + (size_t)(rec_off + j0) * P::RW;
      for (int e = threadIdx.x; e < cnt * P::RW; e += NT) sh[(e % P::RW) * CH + e / P::RW] = src[e];
      for (int q = cnt + threadIdx.x; q < ((cnt + 31) & ~31); q += NT) P::template pad<CH>(sh, q);
      __syncthreads();
      if (j0 < t0 + T)
        sym_chunk<P, TPT, CH, true>(g, tg, idx, acc, sh, cnt, j0, jred);
      else
        sym_chunk<P, TPT, CH, false>(g, tg, idx, acc, sh, cnt, j0, jred);
#pragma unroll
      for (int k = 0; k < TPT; ++k) P::renorm(acc[k]);
      __syncthreads();
      for (int q = threadIdx.x; q < cnt; q += NT) {
        Acc v = jred[0][q];
#pragma unroll
        for (int w = 1; w < NW; ++w) v.p = P::add(v.p, jred[w][q].p), v.q = P::add(v.q, jred[w][q].q);
        const int o = j0 + q - t0;
        part[jrow + o] = P::out(v.p);
        part[jrow + len + o] = P::out(v.q);
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k)
      if (idx[k] < n) {
        part[(size_t)ioff + idx[k] - t0] = P::out(acc[k].p);
        part[(size_t)ioff + T + idx[k] - t0] = P::out(acc[k].q);
      }
  }
}

// ------------------------------------------------------------------ pack / reduce
// Records of every system at vec_off / 2 (RW vectors each).  lay[k] = {geo_off, n, vec_off, chg_off}.
// A u: a = ds psi, alpha = ds phi; A^T w: a = wphi, alpha = wpsi.
// sigma: the positions and alpha are multiplied by it (kappa-scaled records; 1 otherwise)
template <typename V4, typename T>
__global__ void k_pack_sym(const int4* __restrict__ lay, bool transpose, const double4_32a* __restrict__ tgt64,
                           const double* __restrict__ u, V4* __restrict__ rec, const int* __restrict__ skip,
                           int skip_stride, double sigma) {
  chain_wait();
  chain_release();
  const int k = blockIdx.y;
  const int4 L = lay[k];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.y || (skip != nullptr && skip[(size_t)k * skip_stride] != 0)) return;
  const double4_32a g = tgt64[2 * (L.x + j)], v = tgt64[2 * (L.x + j) + 1];
  const double phi = u[L.z + j], psi = u[L.z + L.y + j];
  const double a = transpose ? phi : g.w * psi;
  const double al = sigma * (transpose ? psi : g.w * phi);
  V4 r0, r1;
  r0.x = (T)(sigma * g.x), r0.y = (T)(sigma * g.y), r0.z = (T)(sigma * g.z), r0.w = (T)a;
  r1.x = (T)v.x, r1.y = (T)v.y, r1.z = (T)v.z, r1.w = (T)al;
  V4* o = rec + 2 * (size_t)(L.z / 2 + j);
  o[0] = r0, o[1] = r1;
}

__global__ void k_pack_sym_df(const int4* __restrict__ lay, bool transpose, const double4_32a* __restrict__ tgt64,
                              const double* __restrict__ u, float4* __restrict__ rec, const int* __restrict__ skip,
                              int skip_stride, double sigma) {
  chain_wait();
  chain_release();
  const int k = blockIdx.y;
  const int4 L = lay[k];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.y || (skip != nullptr && skip[(size_t)k * skip_stride] != 0)) return;
  const double4_32a g = tgt64[2 * (L.x + j)], v = tgt64[2 * (L.x + j) + 1];
  const double phi = u[L.z + j], psi = u[L.z + L.y + j];
  const df a = df_from_double(transpose ? phi : g.w * psi);
  const df al = df_from_double(sigma * (transpose ? psi : g.w * phi));
  const df x0 = df_from_double(sigma * g.x), x1 = df_from_double(sigma * g.y), x2 = df_from_double(sigma * g.z);
  const df n0 = df_from_double(v.x), n1 = df_from_double(v.y), n2 = df_from_double(v.z);
  float4* o = rec + 4 * (size_t)(L.z / 2 + j);
  o[0] = make_float4(x0.hi, x1.hi, x2.hi, a.hi);
  o[1] = make_float4(x0.lo, x1.lo, x2.lo, a.lo);
  o[2] = make_float4(n0.hi, n1.hi, n2.hi, al.hi);
  o[3] = make_float4(n0.lo, n1.lo, n2.lo, al.lo);
}

// y_i = diag u_i - (1/(4 pi)) scale_i f_c (i-side blocks of the element's row + j-side rows 0..E),
// f_c = f.x for the phi rows and f.y for the psi rows (the factors of kappa-scaled records).
// tab[k] = {n, first row entry, j-side base, T}; tab[row entry + E] = {first i-side block, blocks, 0, 0}.
template <typename PT>
__global__ void k_reduce_sym(const int4* __restrict__ lay, const int4* __restrict__ tab, const PT* __restrict__ part,
                             const double* __restrict__ u, double* __restrict__ y, double d_phi, double d_psi,
                             const double4_32a* __restrict__ tgt64_for_area, const int* __restrict__ skip,
                             int skip_stride, double2 f) {
  chain_wait();
  chain_release();
  const int k = blockIdx.y;
  const int4 L = lay[k], S = tab[k];
  const int n = L.y, T = S.w;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n || (skip != nullptr && skip[(size_t)k * skip_stride] != 0)) return;
  const int c = i < n ? 0 : 1;
  const int e = i - c * n;
  const int E = e / T;
  const int4 R = tab[S.y + E];
  double acc = 0.0;
  for (int b = 0; b < R.y; ++b) acc += (double)part[(size_t)R.x + (size_t)b * 2 * T + (size_t)c * T + (e - E * T)];
  // rows 0..E in order; four loads in flight at a time
  auto at = [&](int I) {
    const int64_t row = (int64_t)S.z + 2 * ((int64_t)I * n - (int64_t)T * I * (I - 1) / 2);
    return (double)part[row + (int64_t)c * (n - I * T) + (e - I * T)];
  };
  int I = 0;
  for (; I + 4 <= E + 1; I += 4) {
    const double v0 = at(I), v1 = at(I + 1), v2 = at(I + 2), v3 = at(I + 3);
    acc += v0;
    acc += v1;
    acc += v2;
    acc += v3;
  }
  for (; I <= E; ++I) acc += at(I);
  const double sc = tgt64_for_area ? tgt64_for_area[2 * (L.x + e)].w : 1.0;
  y[L.z + i] = (c == 0 ? d_phi : d_psi) * u[L.z + i] - kInv4PiS * sc * (c == 0 ? f.x : f.y) * acc;
}

int blocks_of(int64_t n, int bs) { return (int)std::max<int64_t>(1, (n + bs - 1) / bs); }

// ------------------------------------------------------------------ work list
// Folded rows (I, nT - 1 - I) of every system are cut into pieces of about
// Lsrc sources; Lsrc is the candidate (the length giving 1 .. 32 waves of
// equal pieces) whose greedy schedule (pieces sorted by size, each to the
// first free CTA slot) finishes first.  A piece costs its
// sources plus 32 per segment (loading a tile, storing its partials).
struct HostPlan {
  std::vector<int4> items, tab;
  int n_items = 0;
  int64_t part_len = 0;
};

HostPlan compute_sym_plan(const SysLayout& L, int T, int slots, int ch);

// The work list depends only on the layout, the tile and the CTA slots:
// handles of the same sizes share its host copy (a process-wide memo of at
// most 64 entries), and each uploads it once.
ItemPlan* plan_sym(Surface* s, uint64_t key, const SysLayout& L, int T, int slots, int ch) {
  auto it = s->plans.find(key);
  if (it != s->plans.end()) return it->second.get();
  uint64_t mk = 0xcbf29ce484222325ull;
  auto mix = [&](uint64_t v) { mk = (mk ^ v) * 0x100000001b3ull; };
  mix((uint64_t)T), mix((uint64_t)slots), mix((uint64_t)ch), mix((uint64_t)L.K);
  for (int k = 0; k < L.K; ++k) mix((uint64_t)L.n[k]), mix((uint64_t)L.vec_off[k]);
  static std::mutex mu;
  static std::map<uint64_t, std::shared_ptr<const HostPlan>> memo;
  std::shared_ptr<const HostPlan> hp;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto m = memo.find(mk);
    if (m != memo.end()) hp = m->second;
  }
  if (!hp) {
    hp = std::make_shared<const HostPlan>(compute_sym_plan(L, T, slots, ch));
    std::lock_guard<std::mutex> lock(mu);
    if (memo.size() >= 64) memo.erase(memo.begin());
    memo[mk] = hp;
  }
  auto plan = std::make_unique<ItemPlan>();
  plan->n_items = hp->n_items;
  plan->part_len = hp->part_len;
  plan->items.ensure(hp->items.size(), s->stream);
  plan->tab.ensure(hp->tab.size(), s->stream);
  BIPB_CUDA(cudaMemcpyAsync(plan->items.p, hp->items.data(), hp->items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            s->stream));
  BIPB_CUDA(cudaMemcpyAsync(plan->tab.p, hp->tab.data(), hp->tab.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  ++s->alloc_gen;
  ItemPlan* raw = plan.get();
  s->plans[key] = std::move(plan);
  return raw;
}

HostPlan compute_sym_plan(const SysLayout& L, int T, int slots, int ch) {
  const int K = L.K;
  struct Fold {
    int k, Ia, Ib, la, lb;  // rows Ia and Ib (-1: none) with la and lb sources
  };
  std::vector<Fold> folds;
  int64_t total = 0;
  int n_max = 1;
  for (int k = 0; k < K; ++k) {
    const int n = L.n[k], nT = (n + T - 1) / T;
    n_max = std::max(n_max, n);
    for (int I = 0; I < nT / 2; ++I) {
      const int Ib = nT - 1 - I;
      folds.push_back(Fold{k, I, Ib, n - I * T, n - Ib * T});
    }
    if (nT % 2) folds.push_back(Fold{k, nT / 2, -1, n - (nT / 2) * T, 0});
  }
  for (const Fold& f : folds) total += f.la + f.lb;
  auto pieces_of = [&](const Fold& f, double Ls) {
    return std::max(1, (int)std::lround((f.la + f.lb) / Ls));
  };
  auto makespan = [&](double Ls) {
    std::vector<double> cost;
    for (const Fold& f : folds) {
      const int P = pieces_of(f, Ls), len = f.la + f.lb;
      for (int p = 0; p < P; ++p) {
        const int a = (int)((int64_t)p * len / P), b = (int)((int64_t)(p + 1) * len / P);
        const int segs = (a < f.la ? 1 : 0) + (b > f.la ? 1 : 0);
        cost.push_back((double)(b - a) + 32.0 * segs);
      }
    }
    std::sort(cost.begin(), cost.end(), std::greater<double>());
    std::priority_queue<double, std::vector<double>, std::greater<double>> q;
    for (int i = 0; i < slots; ++i) q.push(0.0);
    double end = 0.0;
    for (double c : cost) {
      const double t = q.top() + c;
      q.pop();
      q.push(t);
      end = std::max(end, t);
    }
    return end;
  };
  // candidates: the piece length that gives w waves of equal pieces, w from 1
  // to 32 (uneven batches need many short pieces to balance); stop once the
  // schedule is within 1 % of the ideal total / slots
  const double ideal = (double)total / (double)slots;
  double best_L = 2.0 * n_max, best = makespan(best_L);
  static const double kWaves[] = {1, 1.5, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  for (double w : kWaves) {
    if (best <= 1.01 * ideal) break;
    const double Ls = std::max((double)ch, (double)total / (w * slots));
    const double m = makespan(Ls);
    if (m < best * 0.995) best = m, best_L = Ls;
  }

  // segments: {k, row, s0, s1, piece}; a piece has one or two
  struct Seg {
    int k, I, s0, s1, piece;
  };
  std::vector<Seg> segs;
  std::vector<int> piece_cost;
  for (const Fold& f : folds) {
    const int P = pieces_of(f, best_L), len = f.la + f.lb;
    for (int p = 0; p < P; ++p) {
      const int a = (int)((int64_t)p * len / P), b = (int)((int64_t)(p + 1) * len / P);
      const int id = (int)piece_cost.size();
      piece_cost.push_back(b - a);
      const int ta = f.Ia * T;
      if (a < f.la) segs.push_back(Seg{f.k, f.Ia, ta + a, ta + std::min(b, f.la), id});
      if (b > f.la) {
        const int tb = f.Ib * T;
        segs.push_back(Seg{f.k, f.Ib, tb + std::max(a - f.la, 0), tb + (b - f.la), id});
      }
    }
  }
  // i-side blocks numbered row by row (system, row, first source)
  std::vector<int> order(segs.size());
  for (size_t i = 0; i < segs.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    const Seg &a = segs[x], &b = segs[y];
    if (a.k != b.k) return a.k < b.k;
    if (a.I != b.I) return a.I < b.I;
    return a.s0 < b.s0;
  });
  std::vector<int> block(segs.size());
  std::vector<int4> tab(K);
  std::vector<int> rowbase(K);
  int nrows = 0;
  for (int k = 0; k < K; ++k) {
    rowbase[k] = K + nrows;
    nrows += (L.n[k] + T - 1) / T;
  }
  std::vector<int4> rowtab(nrows, make_int4(0, 0, 0, 0));
  for (size_t r = 0; r < order.size(); ++r) {
    const Seg& g = segs[order[r]];
    block[order[r]] = (int)r;
    int4& e = rowtab[rowbase[g.k] - K + g.I];
    if (e.y == 0) e.x = (int)((int64_t)r * 2 * T);
    e.y += 1;
  }
  int64_t off = (int64_t)segs.size() * 2 * T;
  std::vector<int64_t> jbase(K);
  for (int k = 0; k < K; ++k) {
    const int n = L.n[k], nT = (n + T - 1) / T;
    jbase[k] = off;
    off += 2 * ((int64_t)nT * n - (int64_t)T * nT * (nT - 1) / 2);
    tab[k] = make_int4(n, rowbase[k], (int)jbase[k], T);
  }
  BIPB_REQUIRE(off < ((int64_t)1 << 31), "mat-vec too large for one symmetric work list");

  // items: three int4 per piece, largest piece first
  const int n_pieces = (int)piece_cost.size();
  std::vector<int4> items((size_t)3 * n_pieces, make_int4(0, 0, 0, 0));
  std::vector<int> nseg(n_pieces, 0);
  for (size_t i = 0; i < segs.size(); ++i) {
    const Seg& g = segs[i];
    const int p = g.piece;
    items[3 * p] = make_int4(L.vec_off[g.k] / 2, L.n[g.k], g.k, (int)jbase[g.k]);
    items[3 * p + 1 + nseg[p]++] = make_int4(g.I * T, g.s0, g.s1, (int)((int64_t)block[i] * 2 * T));
  }
  std::vector<int> porder(n_pieces);
  for (int p = 0; p < n_pieces; ++p) porder[p] = p;
  std::stable_sort(porder.begin(), porder.end(), [&](int x, int y) { return piece_cost[x] > piece_cost[y]; });
  std::vector<int4> sorted((size_t)3 * n_pieces);
  for (int p = 0; p < n_pieces; ++p)
    for (int c = 0; c < 3; ++c) sorted[(size_t)3 * p + c] = items[(size_t)3 * porder[p] + c];
  tab.insert(tab.end(), rowtab.begin(), rowtab.end());
  HostPlan hp;
  hp.items = std::move(sorted);
  hp.tab = std::move(tab);
  hp.n_items = n_pieces;
  hp.part_len = off;
  return hp;
}

// Plan-cache key of one symmetric pass over one layout (SplitMix64 finaliser,
// so that distinct (pass, layout) pairs do not collide by construction).
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
uint64_t sym_key(int pass_id, uint64_t layout_key) {
  return mix64(layout_key ^ mix64(0x5e11000000000000ull + (uint64_t)pass_id));
}

// Partial sums a symmetric pass over L needs with tiles of T targets (the
// i-side blocks excluded), and whether they fit the 32-bit offsets.
bool sym_fits(const SysLayout& L, int T) {
  int64_t off = 0;
  for (int k = 0; k < L.K; ++k) {
    const int n = L.n[k], nT = (n + T - 1) / T;
    off += 2 * ((int64_t)nT * n - (int64_t)T * nT * (nT - 1) / 2);
  }
  return off < ((int64_t)1 << 30);
}

template <class P, int NT, int TPT, int CH, int MINB>
int sym_occupancy() {
  static int occ = [] {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_sym<P, NT, TPT, CH, MINB>, NT, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      o = 1;
    }
    return std::max(o, 1);
  }();
  return occ;
}

template <class P, int NT, int TPT, int CH, int MINB>
void run_sym(Surface* s, int pass_id, int kind, const SysLayout& L, const typename P::Args& g, bool transpose,
             DevBuf<typename P::V4>& recbuf, DevBuf<typename P::PT>& partbuf, const double* u, double* y,
             double dphi, double dpsi, const int* skip, int skip_stride, double sigma = 1.0) {
  constexpr int T = NT * TPT;
  if (!P::SCALED) sigma = 1.0;
  // A u: P ~ sigma, Q ~ sigma^2; A^T w: P ~ sigma^2, Q ~ sigma (pair.cuh)
  const double2 f = transpose ? make_double2(sigma * sigma, sigma) : make_double2(sigma, sigma * sigma);
  const uint64_t key = sym_key(pass_id, L.key);
  ItemPlan* plan = plan_sym(s, key, L, T, s->num_sms * sym_occupancy<P, NT, TPT, CH, MINB>(), CH);
  s->grow(recbuf, (size_t)(L.len / 2) * P::RW);
  s->grow(partbuf, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  if constexpr (std::is_same<typename P::PT, double>::value && std::is_same<typename P::V4, float4>::value) {
    launch_chained(k_pack_sym_df, dim3(blocks_of(L.max_n, 256), L.K), 256, 0, s->stream, lay, transpose, s->tgt64.p, u,
                   recbuf.p, skip, skip_stride, sigma);
  } else {
    launch_chained(k_pack_sym<typename P::V4, typename P::PT>, dim3(blocks_of(L.max_n, 256), L.K), 256, 0, s->stream,
                   lay, transpose, s->tgt64.p, u, recbuf.p, skip, skip_stride, sigma);
  }
  BIPB_LAUNCHED(s);
  {
    TimedLaunch tl(s, kind);
    launch_chained(k_sym<P, NT, TPT, CH, MINB>, plan->n_items, NT, 0, s->stream, g, plan->items.p, recbuf.p,
                   partbuf.p, skip, skip_stride);
    BIPB_LAUNCHED(s);
  }
  launch_chained(k_reduce_sym<typename P::PT>, dim3(blocks_of(2 * (int64_t)L.max_n, 256), L.K), 256, 0, s->stream, lay,
                 plan->tab.p, partbuf.p, u, y, dphi, dpsi, transpose ? s->tgt64.p : nullptr, skip, skip_stride, f);
  BIPB_LAUNCHED(s);
}

}  // namespace

// The symmetric FP32 / FP64 forms: LAPLACE for kappa = 0, kappa-scaled
// records for kappa >= kSymKappaMin; in between (a Debye length above 1e6 A)
// the scaled 1/r^3 could leave the FP32 range, and the caller takes the
// ordered kernels.
constexpr double kSymKappaMin = 1e-6;

template <typename T>
bool sym_form(double kappa, PairConst<T>& c, bool& laplace) {
  laplace = kappa == 0.0;
  if (!laplace && kappa < kSymKappaMin) return false;
  c.smax = (T)(laplace ? kSMaxD : kSMaxD / kappa);  // the 1/r cap at 1e-6 A, in the units of the records
  return true;
}

bool matvec_sym32(Surface* s, const SysLayout& L, const PairConst<float>& c0, double kappa, bool transpose,
                  int variant, const double* u, double* y, double dphi, double dpsi, const int* skip,
                  int skip_stride) {
  static const int kT[3] = {512, 512, 1024};  // NT x TPT of the variants below
  if (variant < 0 || variant > 2) throw Error(BIPB_ERR_INVALID_ARG, "unknown symmetric FP32 mat-vec variant");
  PairConst<float> c = c0;
  bool lap = false;
  if (!sym_fits(L, kT[variant]) || !sym_form(kappa, c, lap)) return false;
  const int kind = transpose ? kTMv32T : kTMv32;
#define BIPB_SYM32_RUN(TR_, LAP_, V_, NT_, TPT_, CH_, MINB_)                                                    \
  run_sym<SymPolicy<float, TR_, LAP_>, NT_, TPT_, CH_, MINB_>(s, (TR_ ? 0x100 : 0x200) + V_, kind, L, {c}, TR_, \
                                                               s->rec32, s->part32, u, y, dphi, dpsi, skip,      \
                                                               skip_stride, kappa)
#define BIPB_SYM32(V_, NT_, TPT_, CH_, MINB_)                     \
  case V_:                                                         \
    if (transpose) {                                               \
      if (lap)                                                     \
        BIPB_SYM32_RUN(true, true, V_, NT_, TPT_, CH_, MINB_);     \
      else                                                         \
        BIPB_SYM32_RUN(true, false, V_, NT_, TPT_, CH_, MINB_);    \
    } else {                                                       \
      if (lap)                                                     \
        BIPB_SYM32_RUN(false, true, V_, NT_, TPT_, CH_, MINB_);    \
      else                                                         \
        BIPB_SYM32_RUN(false, false, V_, NT_, TPT_, CH_, MINB_);   \
    }                                                              \
    return true;
  switch (variant) {
    BIPB_SYM32(0, 256, 2, 64, 4)
    BIPB_SYM32(1, 128, 4, 64, 5)
    BIPB_SYM32(2, 256, 4, 64, 2)
  }
#undef BIPB_SYM32
#undef BIPB_SYM32_RUN
  return false;
}

bool matvec_sym64(Surface* s, const SysLayout& L, const PairConst<double>& c0, double kappa, bool transpose,
                  const double* u, double* y, double dphi, double dpsi, const int* skip, int skip_stride) {
  PairConst<double> c = c0;
  bool lap = false;
  if (!sym_fits(L, 256) || !sym_form(kappa, c, lap)) return false;
#define BIPB_SYM64_RUN(TR_, LAP_)                                                                                \
  run_sym<SymPolicy<double, TR_, LAP_>, 128, 2, 64, 1>(s, TR_ ? 0x300 : 0x400, TR_ ? kTMv64T : kTMv64, L, {c}, TR_, \
                                                      s->rec64, s->part64, u, y, dphi, dpsi, skip, skip_stride,     \
                                                      kappa)
  if (transpose) {
    if (lap)
      BIPB_SYM64_RUN(true, true);
    else
      BIPB_SYM64_RUN(true, false);
  } else {
    if (lap)
      BIPB_SYM64_RUN(false, true);
    else
      BIPB_SYM64_RUN(false, false);
  }
#undef BIPB_SYM64_RUN
  return true;
}

bool matvec_sym_df(Surface* s, const SysLayout& L, const DFConst& c, double kappa, bool transpose, const double* u,
                   double* y, double dphi, double dpsi, const int* skip, int skip_stride) {
  if (!sym_fits(L, 128)) return false;
  // kappa-scaled records for kappa >= kSymKappaMin (the FP32 rule), unscaled otherwise
  const bool scaled = kappa >= kSymKappaMin;
#define BIPB_SYMDF_RUN(TR_, SC_)                                                                                 \
  run_sym<SymDFPolicy<TR_, SC_>, 128, 1, 32, 1>(s, TR_ ? 0x500 : 0x600, TR_ ? kTMvDFT : kTMvDF, L, {c}, TR_,     \
                                               s->recdf, s->part64, u, y, dphi, dpsi, skip, skip_stride, kappa)
  if (transpose) {
    if (scaled)
      BIPB_SYMDF_RUN(true, true);
    else
      BIPB_SYMDF_RUN(true, false);
  } else {
    if (scaled)
      BIPB_SYMDF_RUN(false, true);
    else
      BIPB_SYMDF_RUN(false, false);
  }
#undef BIPB_SYMDF_RUN
  return true;
}

}  // namespace bipb
