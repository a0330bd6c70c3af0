// Pair passes of the direct-sum pipeline (Sec. 2.4): the mat-vec of Eqs. 5-6
// and its transpose, the source term (Eq. for S1, S2), the reaction potential
// and solvation energy (Eq. for E_sol), and the energy gradient.
//
// Every pass has one shape.  A pass runs over K independent systems at once
// (several right-hand sides of one surface, or several surfaces of uneven
// size); its work is a list of items, each one tile of a system's targets
// (several per thread, in registers) against one range of that system's
// sources (streamed through shared memory CH records at a time).  One launch
// covers the whole list; items are balanced in size and their count fills
// whole waves of resident CTAs.  Each item writes per-split partial sums; a
// reduction kernel adds the splits of every target in a fixed order in FP64,
// applies 1/(4 pi) and the diagonal, and writes the output, so every pass is
// bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr double kInv4Pi = 1.0 / (4.0 * kPi);

template <typename T>
struct V4T;
template <>
struct V4T<float> {
  using type = float4;
};
template <>
struct V4T<double> {
  using type = double4_32a;
};

__device__ __forceinline__ bool sys_skipped(const int* skip, int stride, int sys) {
  return skip != nullptr && skip[(size_t)sys * stride] != 0;
}

// ------------------------------------------------------------------ policies
// A policy P describes one pass: the target state loaded into registers, the
// source record (RW vectors of 4), the accumulator (NOUT values) and the pair
// update.  load() takes a global target index; store() writes the NOUT values
// of local target i to part[out + c * n_tgt + i].

template <typename T>
struct ElemTgt {
  T x, y, z, nx, ny, nz;
};

template <typename T, bool TRANS>
struct MatvecPolicy {
  using V4 = typename V4T<T>::type;
  static constexpr int RW = 2;
  static constexpr int NOUT = 2;
  static constexpr bool SELF = true;
  template <class A>
  __device__ static void prologue(const A&) {}
  using Tgt = ElemTgt<T>;
  struct Acc {
    T p, q;
  };
  struct Args {
    const V4* tgt;  // 2 per element: (x, y, z, area), (nx, ny, nz, 0)
    T* part;
    PairConst<T> c;
  };
  __device__ static void load(const Args& a, int i, Tgt& t) {
    V4 g = a.tgt[2 * i], v = a.tgt[2 * i + 1];
    t = Tgt{g.x, g.y, g.z, v.x, v.y, v.z};
  }
  __device__ static void zero(Acc& acc) { acc.p = T(0), acc.q = T(0); }
  __device__ static void renorm(Acc&) {}
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const V4* r, bool self, Acc& acc) {
    const V4 A = r[0], B = r[1];
    if (TRANS)
      pair_transpose<MASK>(t.x, t.y, t.z, t.nx, t.ny, t.nz, A.x, A.y, A.z, A.w, B.x, B.y, B.z, self,
                           a.c, acc.p, acc.q);
    else
      pair_forward<MASK>(t.x, t.y, t.z, t.nx, t.ny, t.nz, A.x, A.y, A.z, A.w, B.x, B.y, B.z, self, a.c,
                         acc.p, acc.q);
  }
  __device__ static void store(const Args& a, int out, int n_tgt, int i, const Acc& acc) {
    a.part[(size_t)out + i] = acc.p;
    a.part[(size_t)out + n_tgt + i] = acc.q;
  }
};

// Mat-vec in double-float arithmetic (df64.cuh).  Record per source, 4 float4:
// (x.hi, a.hi), (x.lo, a.lo), (m.hi, 0), (m.lo, 0) with a = ds psi and
// m = ds phi n (forward) or a = wphi, m = wpsi n (transposed).
__device__ df* df_exp_table() {
  __shared__ __align__(16) df tab[kExpTab];
  return tab;
}

template <bool TRANS>
struct MatvecDFPolicy {
  static constexpr int RW = 4;
  static constexpr int NOUT = 2;
  static constexpr bool SELF = true;
  struct Tgt {
    df x[3], n[3];
  };
  struct Acc {
    df p, q;
  };
  struct Args {
    const double4_32a* tgt;
    double* part;
    DFConst c;
  };
  __device__ static void prologue(const Args& a) {
    df_load_exp_table(df_exp_table(), a.c);
  }
  __device__ static void load(const Args& a, int i, Tgt& t) {
    double4_32a g = a.tgt[2 * i], v = a.tgt[2 * i + 1];
    t.x[0] = df_from_double(g.x), t.x[1] = df_from_double(g.y), t.x[2] = df_from_double(g.z);
    t.n[0] = df_from_double(v.x), t.n[1] = df_from_double(v.y), t.n[2] = df_from_double(v.z);
  }
  __device__ static void zero(Acc& acc) { acc.p = df{0.f, 0.f}, acc.q = df{0.f, 0.f}; }
  __device__ static void renorm(Acc&) {}
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const float4* r, bool self, Acc& acc) {
    const float4 A = r[0], B = r[1], C = r[2], D = r[3];
    const df xs[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    const df m[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
    const df w = df{A.w, B.w};
    if (TRANS)
      df_pair_transpose<MASK>(t.x, t.n, xs, w, m, self, a.c, df_exp_table(), acc.p, acc.q);
    else
      df_pair_forward<MASK>(t.x, t.n, xs, w, m, self, a.c, df_exp_table(), acc.p, acc.q);
  }
  __device__ static void store(const Args& a, int out, int n_tgt, int i, const Acc& acc) {
    a.part[(size_t)out + i] = df_to_double(acc.p);
    a.part[(size_t)out + n_tgt + i] = df_to_double(acc.q);
  }
};

// Source term in df64: target element i, source charge k with df record
// (y_k.hi, q_k.hi), (y_k.lo, q_k.lo), d = x_i - y_k:
//   4 pi eps_in S1 += q s,   4 pi eps_in S2 += -q (n_i.d) s^3   (d/dnu_x = +n_x.grad_x)
// GB300 executes FP64 at 1/64 of the FP32 rate; df64 keeps b accurate to
// about 1e-14 relative at a fraction of the FP64 cost.
struct SourcePolicy {
  static constexpr int RW = 2;
  static constexpr int NOUT = 2;
  static constexpr bool SELF = false;
  template <class A>
  __device__ static void prologue(const A&) {}
  struct Tgt {
    df x[3], n[3];
  };
  struct Acc {
    df s1, s2;
  };
  struct Args {
    const double4_32a* tgt;  // 2 per element
    double* part;
  };
  __device__ static void load(const Args& a, int i, Tgt& t) {
    double4_32a g = a.tgt[2 * i], v = a.tgt[2 * i + 1];
    t.x[0] = df_from_double(g.x), t.x[1] = df_from_double(g.y), t.x[2] = df_from_double(g.z);
    t.n[0] = df_from_double(v.x), t.n[1] = df_from_double(v.y), t.n[2] = df_from_double(v.z);
  }
  __device__ static void zero(Acc& acc) { acc.s1 = df{0.f, 0.f}, acc.s2 = df{0.f, 0.f}; }
  __device__ static void renorm(Acc&) {}
  template <bool MASK>
  __device__ static void pair(const Args&, const Tgt& t, const float4* r, bool, Acc& acc) {
    const float4 A = r[0], B = r[1];
    const df y[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    df_source_pair(t.x, t.n, y, df{A.w, B.w}, acc.s1, acc.s2);
  }
  __device__ static void store(const Args& a, int out, int n_tgt, int i, const Acc& acc) {
    a.part[(size_t)out + i] = df_to_double(acc.s1);
    a.part[(size_t)out + n_tgt + i] = df_to_double(acc.s2);
  }
};

// Reaction potential at a charge y_k from the surface in df64 (forward df
// record (x_j, a_j = ds psi_j), m_j = ds phi_j n_j), d = y_k - x_j:
//   4 pi phi_reac += s [ (1 - e) a_j + (eps t - 1) (m_j.d) s^2 ]  (K1 psi + K2 phi, n_j only)
struct ReactionPolicy {
  static constexpr int RW = 4;
  static constexpr int NOUT = 1;
  static constexpr bool SELF = false;
  struct Tgt {
    df y[3];
  };
  struct Acc {
    df p;
  };
  struct Args {
    const double4_32a* pts;  // (y, q)
    double* part;
    DFConst c;
  };
  template <class A>
  __device__ static void prologue(const A& a) {
    df_load_exp_table(df_exp_table(), a.c);
  }
  __device__ static void load(const Args& a, int k, Tgt& t) {
    double4_32a g = a.pts[k];
    t.y[0] = df_from_double(g.x), t.y[1] = df_from_double(g.y), t.y[2] = df_from_double(g.z);
  }
  __device__ static void zero(Acc& acc) { acc.p = df{0.f, 0.f}; }
  __device__ static void renorm(Acc&) {}
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const float4* r, bool, Acc& acc) {
    const float4 A = r[0], B = r[1], C = r[2], D = r[3];
    const df xs[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    const df m[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
    df_reaction_pair(t.y, xs, df{A.w, B.w}, m, a.c, df_exp_table(), acc.p);
  }
  __device__ static void store(const Args& a, int out, int, int k, const Acc& acc) {
    a.part[(size_t)out + k] = df_to_double(acc.p);
  }
};

// Potential at a point y in the solvent from the surface in df64 (the same
// forward df record as the reaction pass), the exterior representation:
//   4 pi phi(y) += s [ t (m_j.d) s^2 - (1/eps) e a_j ],  d = y - x_j
struct ExteriorPolicy : ReactionPolicy {
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const float4* r, bool, Acc& acc) {
    const float4 A = r[0], B = r[1], C = r[2], D = r[3];
    const df xs[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    const df m[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
    df_exterior_pair(t.y, xs, df{A.w, B.w}, m, a.c, df_exp_table(), acc.p);
  }
};

// Energy row c in df64: target element j, source charge k (df record
// (y_k, q_k)), d = y_k - x_j:
//   4 pi K2(y_k, x_j) = (eps t - 1) (n_j.d) s^3,  4 pi K1(y_k, x_j) = (1 - e) s
struct EnergyRowPolicy {
  static constexpr int RW = 2;
  static constexpr int NOUT = 2;
  static constexpr bool SELF = false;
  struct Tgt {
    df x[3], n[3];
  };
  struct Acc {
    df cphi, cpsi;
  };
  struct Args {
    const double4_32a* tgt;
    double* part;
    DFConst c;
  };
  template <class A>
  __device__ static void prologue(const A& a) {
    df_load_exp_table(df_exp_table(), a.c);
  }
  __device__ static void load(const Args& a, int i, Tgt& t) {
    double4_32a g = a.tgt[2 * i], v = a.tgt[2 * i + 1];
    t.x[0] = df_from_double(g.x), t.x[1] = df_from_double(g.y), t.x[2] = df_from_double(g.z);
    t.n[0] = df_from_double(v.x), t.n[1] = df_from_double(v.y), t.n[2] = df_from_double(v.z);
  }
  __device__ static void zero(Acc& acc) { acc.cphi = df{0.f, 0.f}, acc.cpsi = df{0.f, 0.f}; }
  __device__ static void renorm(Acc& acc) {
    acc.cphi = two_sum(acc.cphi.hi, acc.cphi.lo);
    acc.cpsi = two_sum(acc.cpsi.hi, acc.cpsi.lo);
  }
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const float4* r, bool, Acc& acc) {
    const float4 A = r[0], B = r[1];
    const df y[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    df_energy_row_pair(t.x, t.n, y, df{A.w, B.w}, a.c, df_exp_table(), acc.cphi, acc.cpsi);
  }
  __device__ static void store(const Args& a, int out, int n_tgt, int i, const Acc& acc) {
    a.part[(size_t)out + i] = df_to_double(acc.cphi);
    a.part[(size_t)out + n_tgt + i] = df_to_double(acc.cpsi);
  }
};

// Energy gradient at charge y_k in df64 (df_grad_pair in df64.cuh).  Record
// per element j, 5 float4: (x.hi, a.hi), (x.lo, a.lo), (n.hi, alpha.hi),
// (n.lo, alpha.lo), (lphi.hi, lphi.lo, beta.hi, beta.lo) with a = ds psi,
// alpha = ds phi and the adjoint lam = [lphi; beta].  Outputs per charge: v
// (dE/dq up to 1/2 and 1/(4 pi)) and the three components of the gradient g.
struct GradPolicy {
  static constexpr int RW = 5;
  static constexpr int NOUT = 4;
  static constexpr bool SELF = false;
  struct Tgt {
    df y[3];
  };
  struct Acc {
    df v, g[3];
  };
  struct Args {
    const double4_32a* pts;
    double* part;
    DFConst c;
    df inv_eps_in;
  };
  template <class A>
  __device__ static void prologue(const A& a) {
    df_load_exp_table(df_exp_table(), a.c);
  }
  __device__ static void load(const Args& a, int k, Tgt& t) {
    double4_32a g = a.pts[k];
    t.y[0] = df_from_double(g.x), t.y[1] = df_from_double(g.y), t.y[2] = df_from_double(g.z);
  }
  __device__ static void zero(Acc& acc) {
    acc.v = df{0.f, 0.f};
    for (int m = 0; m < 3; ++m) acc.g[m] = df{0.f, 0.f};
  }
  __device__ static void renorm(Acc& acc) {
    acc.v = two_sum(acc.v.hi, acc.v.lo);
    for (int m = 0; m < 3; ++m) acc.g[m] = two_sum(acc.g[m].hi, acc.g[m].lo);
  }
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const float4* r, bool, Acc& acc) {
    const float4 A = r[0], B = r[1], C = r[2], D = r[3], E = r[4];
    const df x[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    const df nv[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
    df_grad_pair(t.y, x, df{A.w, B.w}, nv, df{C.w, D.w}, df{E.x, E.y}, df{E.z, E.w}, a.c, a.inv_eps_in,
                 df_exp_table(), acc.v, acc.g);
  }
  __device__ static void store(const Args& a, int out, int n_tgt, int k, const Acc& acc) {
    double* o = a.part + (size_t)out + k;
    o[0] = df_to_double(acc.v);
    for (int m = 0; m < 3; ++m) o[(size_t)(1 + m) * n_tgt] = df_to_double(acc.g[m]);
  }
};

// ------------------------------------------------------------------ item kernel
// One CTA per work item (two int4):
//   {tgt_off, n_tgt, t0, sys}  targets tgt_off + [t0, t0 + NT*TPT) of a system
//                              with n_tgt targets (thread t owns t0 + k*NT + t)
//   {src_off, s0, s1, out}     sources src_off + [s0, s1); partials at part[out]
// The self pair (same local index) is masked only in source chunks that
// overlap the item's own targets.
template <class P, typename V4, int NT, int TPT, int CH>
__global__ void __launch_bounds__(NT) k_items(typename P::Args a, const int4* __restrict__ items,
                                              const V4* __restrict__ rec, const int* __restrict__ skip,
                                              int skip_stride) {
  __shared__ V4 sh[CH * P::RW];
  const int4 I0 = items[2 * blockIdx.x], I1 = items[2 * blockIdx.x + 1];
  const int tgt_off = I0.x, n_tgt = I0.y, t0 = I0.z, sys = I0.w;
  const int src_off = I1.x, s0 = I1.y, s1 = I1.z, out = I1.w;
  if (sys_skipped(skip, skip_stride, sys)) return;
  P::prologue(a);  // per-CTA shared tables (made visible by the first barrier below)
  typename P::Tgt tg[TPT];
  typename P::Acc acc[TPT];
  int idx[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    idx[k] = t0 + k * NT + threadIdx.x;
    P::load(a, tgt_off + min(idx[k], n_tgt - 1), tg[k]);
    P::zero(acc[k]);
  }
  for (int j0 = s0; j0 < s1; j0 += CH) {
    const int cnt = min(CH, s1 - j0);
    __syncthreads();
    const V4* src = rec + (size_t)(src_off + j0) * P::RW;
    for (int q = threadIdx.x; q < cnt * P::RW; q += NT) sh[q] = src[q];
    __syncthreads();
    const bool diag = P::SELF && (j0 < t0 + NT * TPT) && (j0 + cnt > t0);
    if (!diag) {
      if (cnt == CH) {
#pragma unroll 2
        for (int jj = 0; jj < CH; ++jj) {
#pragma unroll
          for (int k = 0; k < TPT; ++k) P::template pair<false>(a, tg[k], sh + jj * P::RW, false, acc[k]);
        }
      } else {
        for (int jj = 0; jj < cnt; ++jj) {
#pragma unroll
          for (int k = 0; k < TPT; ++k) P::template pair<false>(a, tg[k], sh + jj * P::RW, false, acc[k]);
        }
      }
    } else {
      for (int jj = 0; jj < cnt; ++jj) {
#pragma unroll
        for (int k = 0; k < TPT; ++k)
          P::template pair<true>(a, tg[k], sh + jj * P::RW, j0 + jj == idx[k], acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) P::renorm(acc[k]);  // lazily updated accumulators back to normal form
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k)
    if (idx[k] < n_tgt) P::store(a, out, n_tgt, idx[k], acc[k]);
}

// ------------------------------------------------------------------ work lists
// Per-system description of one pass: targets [tgt_off, tgt_off + n_tgt),
// sources [src_off, src_off + n_src).
struct PassSys {
  int tgt_off, n_tgt, src_off, n_src;
};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
  return h;
}

// Build (or fetch) the work list of a pass.  Every system's sources are cut
// into splits of about L sources; L is chosen so that the item count fills
// whole waves of resident CTAs (slots = SMs x CTAs per SM) as closely as
// possible, with at least min_src sources per split.  Items are ordered
// largest system first.
ItemPlan* plan_items(Surface* s, int pass_id, const std::vector<PassSys>& sys, int targets_per_cta, int slots,
                     int min_src, int nout) {
  uint64_t key = 0xcbf29ce484222325ull;
  int hdr[4] = {pass_id, targets_per_cta, slots, min_src};
  key = fnv(key, hdr, sizeof(hdr));
  key = fnv(key, sys.data(), sys.size() * sizeof(PassSys));
  auto it = s->plans.find(key);
  if (it != s->plans.end()) return it->second.get();

  const int K = (int)sys.size();
  int n_src_max = 1;
  for (auto& p : sys) n_src_max = std::max(n_src_max, p.n_src);
  auto tiles_of = [&](const PassSys& p) { return (p.n_tgt + targets_per_cta - 1) / targets_per_cta; };
  auto splits_of = [&](const PassSys& p, int L) { return std::max(1, (p.n_src + L - 1) / L); };
  auto count = [&](int L) {
    long c = 0;
    for (auto& p : sys) c += (long)tiles_of(p) * splits_of(p, L);
    return c;
  };
  auto eff = [&](int L) {
    const long c = count(L);
    const long waves = (c + slots - 1) / slots;
    return (double)c / ((double)waves * slots);
  };
  const int max_s = std::max(1, std::min(n_src_max / std::max(min_src, 1), 4096));
  double best = 0.0;
  for (int S = 1; S <= max_s; ++S) best = std::max(best, eff((n_src_max + S - 1) / S));
  int L = n_src_max;
  for (int S = 1; S <= max_s; ++S) {
    const int l = (n_src_max + S - 1) / S;
    if (eff(l) >= 0.98 * best) {  // the fewest splits within 2 % of the best fill
      L = l;
      break;
    }
  }

  auto plan = std::make_unique<ItemPlan>();
  std::vector<int> order(K);
  for (int k = 0; k < K; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long)sys[x].n_tgt * sys[x].n_src > (long)sys[y].n_tgt * sys[y].n_src;
  });
  std::vector<int64_t> sys_out(K);
  std::vector<int> sys_splits(K);
  int64_t out = 0;
  for (int k = 0; k < K; ++k) {
    sys_out[k] = out;
    sys_splits[k] = splits_of(sys[k], L);
    out += (int64_t)sys_splits[k] * nout * sys[k].n_tgt;
  }
  BIPB_REQUIRE(out < ((int64_t)1 << 31), "pass too large for one work list");
  plan->part_len = out;
  std::vector<int4> items;
  for (int k : order) {
    const PassSys& p = sys[k];
    const int S = sys_splits[k];
    for (int t = 0; t < tiles_of(p); ++t)
      for (int sp = 0; sp < S; ++sp) {
        const int s0 = (int)((int64_t)sp * p.n_src / S), s1 = (int)((int64_t)(sp + 1) * p.n_src / S);
        items.push_back(make_int4(p.tgt_off, p.n_tgt, t * targets_per_cta, k));
        items.push_back(make_int4(p.src_off, s0, s1, (int)(sys_out[k] + (int64_t)sp * nout * p.n_tgt)));
      }
  }
  plan->n_items = (int)(items.size() / 2);
  // per-system table for the reductions: {n_tgt, splits, out offset, unused}
  std::vector<int4> tab(K);
  for (int k = 0; k < K; ++k) tab[k] = make_int4(sys[k].n_tgt, sys_splits[k], (int)sys_out[k], 0);
  plan->items.ensure(items.size(), s->stream);
  plan->tab.ensure(K, s->stream);
  BIPB_CUDA(cudaMemcpyAsync(plan->items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            s->stream));
  BIPB_CUDA(cudaMemcpyAsync(plan->tab.p, tab.data(), K * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));  // the host vectors go out of scope
  ++s->alloc_gen;
  ItemPlan* raw = plan.get();
  s->plans[key] = std::move(plan);
  return raw;
}

// Resident CTAs per SM of one item-kernel instantiation (queried once).
template <class P, typename V4, int NT, int TPT, int CH>
int items_occupancy() {
  static int occ = [] {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_items<P, V4, NT, TPT, CH>, NT, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      o = 1;
    }
    return std::max(o, 1);
  }();
  return occ;
}

template <class P, typename V4, int NT, int TPT, int CH>
ItemPlan* plan_pass(Surface* s, int pass_id, const std::vector<PassSys>& sys, int min_src) {
  return plan_items(s, pass_id, sys, NT * TPT, s->num_sms * items_occupancy<P, V4, NT, TPT, CH>(), min_src,
                    P::NOUT);
}

template <class P, typename V4, int NT, int TPT, int CH>
void launch_items(Surface* s, int kind, const ItemPlan* plan, const typename P::Args& a, const V4* rec,
                  const int* skip, int skip_stride) {
  TimedLaunch tlaunch(s, kind);
  k_items<P, V4, NT, TPT, CH><<<plan->n_items, NT, 0, s->stream>>>(a, plan->items.p, rec, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

// ------------------------------------------------------------------ pack / reduce
// grid = (blocks over the largest system, K).  lay[k] = {geo_off, n, vec_off, chg_off}.
// Forward record of element j from u = [phi; psi]: (x, a = ds psi), (m = ds phi n, 0);
// transposed record from w = [wphi; wpsi]: (x, wphi), (p = wpsi n, 0).
// Records of system k start at vec_off / 2.
template <typename V4, typename T>
__global__ void k_pack(const int4* __restrict__ lay, bool transpose, const double4_32a* __restrict__ tgt64,
                       const double* __restrict__ u, V4* __restrict__ rec, const int* __restrict__ skip,
                       int skip_stride) {
  const int k = blockIdx.y;
  const int4 L = lay[k];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.y || sys_skipped(skip, skip_stride, k)) return;
  const double4_32a g = tgt64[2 * (L.x + j)], v = tgt64[2 * (L.x + j) + 1];
  const double* uk = u + L.z;
  const double phi = uk[j], psi = uk[L.y + j];
  const double sc = transpose ? phi : g.w * psi;  // 4th slot
  const double f = transpose ? psi : g.w * phi;   // multiplies the normal
  V4 r0, r1;
  r0.x = (T)g.x, r0.y = (T)g.y, r0.z = (T)g.z, r0.w = (T)sc;
  r1.x = (T)(f * v.x), r1.y = (T)(f * v.y), r1.z = (T)(f * v.z), r1.w = (T)0;
  const size_t o = (size_t)(L.z / 2 + j);
  rec[2 * o] = r0;
  rec[2 * o + 1] = r1;
}

// df64 records (4 float4 per element) of every system, forward or transposed.
__global__ void k_pack_df(const int4* __restrict__ lay, bool transpose, const double4_32a* __restrict__ tgt64,
                          const double* __restrict__ u, float4* __restrict__ rec, const int* __restrict__ skip,
                          int skip_stride) {
  const int k = blockIdx.y;
  const int4 L = lay[k];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.y || sys_skipped(skip, skip_stride, k)) return;
  const double4_32a g = tgt64[2 * (L.x + j)], v = tgt64[2 * (L.x + j) + 1];
  const double* uk = u + L.z;
  const double phi = uk[j], psi = uk[L.y + j];
  const double sc = transpose ? phi : g.w * psi;
  const double f = transpose ? psi : g.w * phi;
  const df x0 = df_from_double(g.x), x1 = df_from_double(g.y), x2 = df_from_double(g.z), w = df_from_double(sc);
  const df m0 = df_from_double(f * v.x), m1 = df_from_double(f * v.y), m2 = df_from_double(f * v.z);
  const size_t o = 4 * (size_t)(L.z / 2 + j);
  rec[o] = make_float4(x0.hi, x1.hi, x2.hi, w.hi);
  rec[o + 1] = make_float4(x0.lo, x1.lo, x2.lo, w.lo);
  rec[o + 2] = make_float4(m0.hi, m1.hi, m2.hi, 0.f);
  rec[o + 3] = make_float4(m0.lo, m1.lo, m2.lo, 0.f);
}

// y_i = diag * u_i - (1/(4 pi)) * scale_i * sum over splits, i < 2n of each system;
// diag = 1/2 (1 + eps) on the phi half and 1/2 (1 + 1/eps) on the psi half;
// scale_i = area of element (i mod n) for the transpose, 1 otherwise.
template <typename PT>
__global__ void k_reduce_matvec(const int4* __restrict__ lay, const int4* __restrict__ tab,
                                const PT* __restrict__ part, const double* __restrict__ u, double* __restrict__ y,
                                double d_phi, double d_psi, const double4_32a* __restrict__ tgt64_for_area,
                                const int* __restrict__ skip, int skip_stride) {
  const int k = blockIdx.y;
  const int4 L = lay[k], T = tab[k];
  const int n = L.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n || sys_skipped(skip, skip_stride, k)) return;
  double acc = 0.0;
  for (int sp = 0; sp < T.y; ++sp) acc += (double)part[(size_t)T.z + (size_t)sp * 2 * n + i];
  const int e = i < n ? i : i - n;
  const double sc = tgt64_for_area ? tgt64_for_area[2 * (L.x + e)].w : 1.0;
  y[L.z + i] = (i < n ? d_phi : d_psi) * u[L.z + i] - kInv4Pi * sc * acc;
}

// b of every system: S1, S2 times 1/(4 pi eps_in)
__global__ void k_reduce_source(const int4* __restrict__ lay, const int4* __restrict__ tab,
                                const double* __restrict__ part, double scale, double* __restrict__ b) {
  const int k = blockIdx.y;
  const int4 L = lay[k], T = tab[k];
  const int n = L.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  double acc = 0.0;
  for (int sp = 0; sp < T.y; ++sp) acc += part[(size_t)T.z + (size_t)sp * 2 * n + i];
  b[L.z + i] = scale * acc;
}

// One block per system: phi_reac_k = (1/(4 pi)) sum over splits;
// E = KCAL/2 sum_k q_k phi_reac_k in a fixed order.
__global__ void k_reduce_reaction(const int4* __restrict__ tab, const int4* __restrict__ lay,
                                  const double* __restrict__ part, const double4_32a* __restrict__ chg,
                                  double* __restrict__ phi_reac, double* __restrict__ e_out) {
  __shared__ double red[1024];
  const int k = blockIdx.x;
  const int4 T = tab[k];
  const int nc = T.x, c0 = lay[k].w;
  double local = 0.0;
  for (int q = threadIdx.x; q < nc; q += blockDim.x) {
    double acc = 0.0;
    for (int sp = 0; sp < T.y; ++sp) acc += part[(size_t)T.z + (size_t)sp * nc + q];
    acc *= kInv4Pi;
    if (phi_reac) phi_reac[c0 + q] = acc;
    local += chg[c0 + q].w * acc;
  }
  red[threadIdx.x] = local;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && e_out) e_out[k] = 0.5 * kKcal * red[0];
}

// Potential at points: out[k n_pts + q] (+)= scale * sum over splits of
// part[tab[k].z + sp * stride * n_pts + q], splits added in order.
__global__ void k_reduce_points(const int4* __restrict__ tab, const double* __restrict__ part, int n_pts,
                                int stride, double scale, int accumulate, double* __restrict__ out) {
  const int k = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_pts) return;
  const int4 T = tab[k];
  double acc = 0.0;
  for (int sp = 0; sp < T.y; ++sp) acc += part[(size_t)T.z + (size_t)sp * stride * n_pts + q];
  double* o = out + (size_t)k * n_pts + q;
  *o = (accumulate ? *o : 0.0) + scale * acc;
}

// Coulomb energy of the charges of system k in the solute, Eq. free_energy
// without the self terms: part[k * gridDim.x + b] = sum over the block's
// charges c of q_c sum_{l != c} q_l / |y_c - y_l| (FP64, l in order, then a
// fixed-order tree over the block).
__global__ void k_coulomb(const int4* __restrict__ lay, const double4_32a* __restrict__ chg,
                          double* __restrict__ part) {  // lay[k] = {0, 0, nc, chg_off}
  __shared__ double red[256];
  const int k = blockIdx.y;
  const int c0 = lay[k].w, nc = lay[k].z;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < nc) {
    const double4_32a a = chg[c0 + c];
    double row = 0.0;
    for (int l = 0; l < nc; ++l) {
      if (l == c) continue;
      const double4_32a b = chg[c0 + l];
      const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
      row += b.w * rsqrt(dx * dx + dy * dy + dz * dz);
    }
    v = a.w * row;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_energy_row_reduce(const int4* __restrict__ lay, const int4* __restrict__ tab,
                                    const double* __restrict__ part, const double4_32a* __restrict__ tgt64,
                                    double* __restrict__ c) {
  const int k = blockIdx.y;
  const int4 L = lay[k], T = tab[k];
  const int n = L.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  double acc = 0.0;
  for (int sp = 0; sp < T.y; ++sp) acc += part[(size_t)T.z + (size_t)sp * 2 * n + i];
  const int e = i < n ? i : i - n;
  c[L.z + i] = tgt64[2 * (L.x + e)].w * kInv4Pi * acc;
}

// Gradient records of every system in df64 (5 float4 per element, at
// vec_off / 2): (x, a = ds psi), (n, alpha = ds phi), (lphi, beta = lpsi).
__global__ void k_pack_grad(const int4* __restrict__ lay, const double4_32a* __restrict__ tgt64,
                            const double* __restrict__ u, const double* __restrict__ lam,
                            float4* __restrict__ rec) {
  const int k = blockIdx.y;
  const int4 L = lay[k];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.y) return;
  const double4_32a g = tgt64[2 * (L.x + j)], v = tgt64[2 * (L.x + j) + 1];
  const double* uk = u + L.z;
  const double* lk = lam + L.z;
  const df x0 = df_from_double(g.x), x1 = df_from_double(g.y), x2 = df_from_double(g.z);
  const df n0 = df_from_double(v.x), n1 = df_from_double(v.y), n2 = df_from_double(v.z);
  const df a = df_from_double(g.w * uk[L.y + j]), al = df_from_double(g.w * uk[j]);
  const df lphi = df_from_double(lk[j]), beta = df_from_double(lk[L.y + j]);
  float4* o = rec + 5 * (size_t)(L.z / 2 + j);
  o[0] = make_float4(x0.hi, x1.hi, x2.hi, a.hi);
  o[1] = make_float4(x0.lo, x1.lo, x2.lo, a.lo);
  o[2] = make_float4(n0.hi, n1.hi, n2.hi, al.hi);
  o[3] = make_float4(n0.lo, n1.lo, n2.lo, al.lo);
  o[4] = make_float4(lphi.hi, lphi.lo, beta.hi, beta.lo);
}

// dE/dq = 1/2 (1/(4 pi)) v and dE/dy = 1/2 q (1/(4 pi)) g per charge (sums over splits in a fixed order)
__global__ void k_reduce_grad(const int4* __restrict__ tab, const int4* __restrict__ lay,
                              const double* __restrict__ part, const double4_32a* __restrict__ chg,
                              double* __restrict__ dq, double* __restrict__ dy) {
  const int k = blockIdx.y;
  const int4 T = tab[k];
  const int nc = T.x, c0 = lay[k].w;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nc) return;
  double v[4] = {0, 0, 0, 0};
  for (int sp = 0; sp < T.y; ++sp)
    for (int c = 0; c < 4; ++c) v[c] += part[(size_t)T.z + (size_t)sp * 4 * nc + (size_t)c * nc + q];
  const double qq = chg[c0 + q].w;
  dq[c0 + q] = 0.5 * kInv4Pi * v[0];
  for (int m = 0; m < 3; ++m) dy[3 * (c0 + q) + m] = 0.5 * qq * kInv4Pi * v[1 + m];
}

template <typename T>
PairConst<T> pair_const(const bipb_medium& m) {
  double eps = m.eps_out / m.eps_in;
  PairConst<T> c;
  c.eps = (T)eps;
  c.inveps = (T)(1.0 / eps);
  c.kappa = (T)m.kappa;
  c.nkl2e = (T)(-m.kappa * 1.4426950408889634);
  c.smax = (T)kSMaxD;
  return c;
}

int blocks_for(int64_t n, int bs) { return (int)std::max<int64_t>(1, (n + bs - 1) / bs); }

enum PassId { kPassMv64 = 1, kPassMv64T, kPassMvDF, kPassMvDFT, kPassMv32 = 16, kPassMv32T = 32, kPassSource = 48,
              kPassReaction, kPassRow, kPassGrad, kPassPotIn, kPassPotOut, kPassPotSrc };

DFConst df_const_impl(const Surface* s, const bipb_medium& m) {
  auto split = [](double v) {
    df r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
  };
  const double eps = m.eps_out / m.eps_in;
  DFConst c;
  c.eps = split(eps);
  c.inveps = split(1.0 / eps);
  c.kappa = split(m.kappa);
  const double L = 0.693147180559945309417232121458 / kExpTab;
  const double l1 = std::ldexp(std::nearbyint(std::ldexp(L, 17)), -17);  // 7 significant bits
  c.l1 = (float)l1;
  c.l2 = (float)(L - l1);
  c.l3 = (float)(L - l1 - (double)c.l2);
  c.inv_l = (float)(kExpTab / 0.693147180559945309417232121458);
  c.tab = s->exptab.p;
  return c;
}

std::vector<PassSys> matvec_sys(const SysLayout& L) {
  std::vector<PassSys> v(L.K);
  for (int k = 0; k < L.K; ++k) v[k] = PassSys{L.geo_off[k], L.n[k], L.vec_off[k] / 2, L.n[k]};
  return v;
}

// FP32 forward / transpose mat-vec (one variant of the autotuned tiling).
template <bool TRANS, int NT, int TPT, int CH>
void run_matvec32(Surface* s, const SysLayout& L, const PairConst<float>& c, const double* u, double* y,
                  double dphi, double dpsi, const int* skip, int skip_stride) {
  using P = MatvecPolicy<float, TRANS>;
  ItemPlan* plan =
      plan_pass<P, float4, NT, TPT, CH>(s, (TRANS ? kPassMv32T : kPassMv32) + s->mv32_variant, matvec_sys(L), CH);
  s->grow(s->rec32, (size_t)L.len);  // 2 records per element = one per unknown
  s->grow(s->part32, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  k_pack<float4, float><<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(
      lay, TRANS, s->tgt64.p, u, s->rec32.p, skip, skip_stride);
  BIPB_LAUNCHED(s);
  typename P::Args a{s->tgt32.p, s->part32.p, c};
  launch_items<P, float4, NT, TPT, CH>(s, TRANS ? kTMv32T : kTMv32, plan, a, s->rec32.p, skip, skip_stride);
  k_reduce_matvec<float><<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      lay, plan->tab.p, s->part32.p, u, y, dphi, dpsi, TRANS ? s->tgt64.p : nullptr, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

template <bool TRANS>
void run_matvec64(Surface* s, const SysLayout& L, const PairConst<double>& c, const double* u, double* y,
                  double dphi, double dpsi, const int* skip, int skip_stride) {
  constexpr int NT = 128, TPT = 2, CH = 64;
  using P = MatvecPolicy<double, TRANS>;
  ItemPlan* plan = plan_pass<P, double4_32a, NT, TPT, CH>(s, TRANS ? kPassMv64T : kPassMv64, matvec_sys(L), CH);
  s->grow(s->rec64, (size_t)L.len);
  s->grow(s->part64, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  k_pack<double4_32a, double><<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(
      lay, TRANS, s->tgt64.p, u, s->rec64.p, skip, skip_stride);
  BIPB_LAUNCHED(s);
  typename P::Args a{s->tgt64.p, s->part64.p, c};
  launch_items<P, double4_32a, NT, TPT, CH>(s, TRANS ? kTMv64T : kTMv64, plan, a, s->rec64.p, skip, skip_stride);
  k_reduce_matvec<double><<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      lay, plan->tab.p, s->part64.p, u, y, dphi, dpsi, TRANS ? s->tgt64.p : nullptr, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

template <bool TRANS>
void run_matvec_df(Surface* s, const SysLayout& L, const DFConst& c, const double* u, double* y, double dphi,
                   double dpsi, const int* skip, int skip_stride) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  using P = MatvecDFPolicy<TRANS>;
  ItemPlan* plan = plan_pass<P, float4, NT, TPT, CH>(s, TRANS ? kPassMvDFT : kPassMvDF, matvec_sys(L), CH);
  s->grow(s->recdf, (size_t)2 * L.len);  // 4 float4 per element
  s->grow(s->part64, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  k_pack_df<<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(lay, TRANS, s->tgt64.p, u, s->recdf.p, skip,
                                                                        skip_stride);
  BIPB_LAUNCHED(s);
  typename P::Args a{s->tgt64.p, s->part64.p, c};
  launch_items<P, float4, NT, TPT, CH>(s, TRANS ? kTMvDFT : kTMvDF, plan, a, s->recdf.p, skip, skip_stride);
  k_reduce_matvec<double><<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      lay, plan->tab.p, s->part64.p, u, y, dphi, dpsi, TRANS ? s->tgt64.p : nullptr, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

__global__ void k_fill_test_vector(int len, double* u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) u[i] = 0.5 + 0.25 * sin(0.37 * i) + (i & 7) * 0.01;
}

}  // namespace

// ------------------------------------------------------------------ layouts
SysLayout make_layout(const std::vector<int>& geo_off, const std::vector<int>& n, const std::vector<int>& chg_off,
                      const std::vector<int>& nc) {
  SysLayout L;
  L.K = (int)n.size();
  L.geo_off = geo_off;
  L.n = n;
  L.chg_off = chg_off;
  L.nc = nc;
  L.vec_off.resize(L.K);
  int64_t off = 0;
  for (int k = 0; k < L.K; ++k) {
    L.vec_off[k] = (int)off;
    off += 2 * (int64_t)n[k];
    L.max_n = std::max(L.max_n, n[k]);
    L.max_nc = std::max(L.max_nc, nc[k]);
  }
  BIPB_REQUIRE(off < ((int64_t)1 << 31), "too many unknowns in one batch");
  L.len = off;
  uint64_t h = 0xcbf29ce484222325ull;
  h = fnv(h, L.geo_off.data(), L.K * sizeof(int));
  h = fnv(h, L.n.data(), L.K * sizeof(int));
  h = fnv(h, L.chg_off.data(), L.K * sizeof(int));
  h = fnv(h, L.nc.data(), L.K * sizeof(int));
  L.key = h;
  return L;
}

const int4* Surface::lay_dev(const SysLayout& L) {
  auto it = layouts.find(L.key);
  if (it != layouts.end()) return it->second->p;
  std::vector<int4> tab(L.K);
  for (int k = 0; k < L.K; ++k) tab[k] = make_int4(L.geo_off[k], L.n[k], L.vec_off[k], L.chg_off[k]);
  auto d = std::make_unique<DevBuf<int4>>();
  d->ensure(L.K, stream);
  BIPB_CUDA(cudaMemcpyAsync(d->p, tab.data(), L.K * sizeof(int4), cudaMemcpyHostToDevice, stream));
  BIPB_CUDA(cudaStreamSynchronize(stream));
  ++alloc_gen;
  const int4* p = d->p;
  layouts[L.key] = std::move(d);
  return p;
}

// ------------------------------------------------------------------ passes
void matvec(Surface* s, const SysLayout& L, const bipb_medium& m, int precision, bool transpose, const double* u,
            double* y, const int* skip, int skip_stride) {
  const double eps = m.eps_out / m.eps_in;
  const double dphi = 0.5 * (1.0 + eps), dpsi = 0.5 * (1.0 + 1.0 / eps);
  if (precision == BIPB_TENSOR) {
    matvec_tc(s, L, pair_const<float>(m), transpose, u, y, dphi, dpsi, skip, skip_stride);
    return;
  }
  if (precision == BIPB_TREE32) {
    matvec_tree(s, L, pair_const<float>(m), transpose, u, y, dphi, dpsi, skip, skip_stride);
    return;
  }
  if (precision == BIPB_DF64) {
    DFConst c = df_const_impl(s, m);
    bool shared_surface = L.K >= 4;
    for (int k = 0; k < L.K && shared_surface; ++k)
      shared_surface = L.geo_off[k] == 0 && L.n[k] == L.n[0] && L.vec_off[k] == 2 * L.n[0] * k;
    if (shared_surface && (!transpose || s->tcx_enabled)) {  // kernel blocks shared by the right-hand sides
      matvec_df_mrhs(s, L, c, transpose, u, y, dphi, dpsi, skip, skip_stride);
      return;
    }
    if (s->sym_pairs && matvec_sym_df(s, L, c, m.kappa, transpose, u, y, dphi, dpsi, skip, skip_stride)) return;
    if (transpose)
      run_matvec_df<true>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);
    else
      run_matvec_df<false>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);
    return;
  }
  if (precision == BIPB_FP64) {
    PairConst<double> c = pair_const<double>(m);
    if (s->sym_pairs && matvec_sym64(s, L, c, m.kappa, transpose, u, y, dphi, dpsi, skip, skip_stride)) return;
    if (transpose)
      run_matvec64<true>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);
    else
      run_matvec64<false>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);
    return;
  }
  PairConst<float> c = pair_const<float>(m);
  int variant = s->mv32_variant;
  if (variant >= kFirstSymVariant) {
    if (matvec_sym32(s, L, c, m.kappa, transpose, variant - kFirstSymVariant, u, y, dphi, dpsi, skip, skip_stride))
      return;
    variant = 0;  // too large for the symmetric work list
  }
  switch (variant) {
#define BIPB_MV32(I_, NT_, TPT_, CH_)                                                      \
  case I_:                                                                                 \
    if (transpose)                                                                         \
      run_matvec32<true, NT_, TPT_, CH_>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);    \
    else                                                                                   \
      run_matvec32<false, NT_, TPT_, CH_>(s, L, c, u, y, dphi, dpsi, skip, skip_stride);   \
    return;
    BIPB_MV32(0, 256, 2, 128)
    BIPB_MV32(1, 256, 1, 128)
    BIPB_MV32(2, 128, 2, 128)
    BIPB_MV32(3, 256, 4, 128)
    BIPB_MV32(4, 128, 4, 64)
    BIPB_MV32(5, 512, 1, 128)
    BIPB_MV32(6, 256, 2, 64)
#undef BIPB_MV32
    default:
      throw Error(BIPB_ERR_INVALID_ARG, "unknown FP32 mat-vec variant");
  }
}


void launch_reduce_matvec64(Surface* s, const SysLayout& L, const int4* tab, const double* part, const double* u,
                            double* y, double dphi, double dpsi, const int* skip, int skip_stride) {
  k_reduce_matvec<double><<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      s->lay_dev(L), tab, part, u, y, dphi, dpsi, nullptr, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

void launch_reduce_matvec32(Surface* s, const SysLayout& L, const int4* tab, const float* part, const double* u,
                            double* y, double dphi, double dpsi, const int* skip, int skip_stride) {
  k_reduce_matvec<float><<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      s->lay_dev(L), tab, part, u, y, dphi, dpsi, nullptr, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

void check_tc_error(Surface* s) {
  if (s->tc_err.cap == 0) return;
  int h = 0;
  BIPB_CUDA(cudaMemcpyAsync(&h, s->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  if (h) {
    BIPB_CUDA(cudaMemsetAsync(s->tc_err.p, 0, sizeof(int), s->stream));
    throw Error(BIPB_ERR_CUDA, "tensor-core mat-vec: a bounded wait on an mbarrier ran out");
  }
}

int autotune_matvec32(Surface* s, const SysLayout& L, const bipb_medium& m, int reps, double* best_ms) {
  const int len = (int)L.len;
  DevBuf<double> u, y;
  u.ensure(len, s->stream);
  y.ensure(len, s->stream);
  k_fill_test_vector<<<blocks_for(len, 256), 256, 0, s->stream>>>(len, u.p);
  BIPB_LAUNCHED(s);
  cudaEvent_t a, b;
  BIPB_CUDA(cudaEventCreate(&a));
  BIPB_CUDA(cudaEventCreate(&b));
  const bool timer_was_on = s->timer.on;
  s->timer.on = false;
  int best = s->mv32_variant;
  double best_t = 1e300;
  try {
    for (int v = 0; v < kNumMv32Variants; ++v) {
      s->mv32_variant = v;
      matvec(s, L, m, BIPB_FP32, false, u.p, y.p, nullptr, 0);  // warm-up (and buffer growth)
      BIPB_CUDA(cudaEventRecord(a, s->stream));
      for (int r = 0; r < reps; ++r) matvec(s, L, m, BIPB_FP32, false, u.p, y.p, nullptr, 0);
      BIPB_CUDA(cudaEventRecord(b, s->stream));
      BIPB_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      BIPB_CUDA(cudaEventElapsedTime(&ms, a, b));
      if (ms < best_t) best_t = ms, best = v;
    }
  } catch (...) {
    s->timer.on = timer_was_on;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  s->timer.on = timer_was_on;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  s->mv32_variant = best;
  if (best_ms) *best_ms = best_t / reps;
  return best;
}

// df64 records of every charge: (y.hi, q.hi), (y.lo, q.lo)
__global__ void k_pack_chg_df(int n_chg, const double4_32a* __restrict__ chg, float4* __restrict__ rec) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_chg) return;
  const double4_32a c = chg[k];
  const df x = df_from_double(c.x), y = df_from_double(c.y), z = df_from_double(c.z), q = df_from_double(c.w);
  rec[2 * k] = make_float4(x.hi, y.hi, z.hi, q.hi);
  rec[2 * k + 1] = make_float4(x.lo, y.lo, z.lo, q.lo);
}

void source_pass(Surface* s, const SysLayout& L, const bipb_medium& m, double* b) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  std::vector<PassSys> sys(L.K);
  int n_chg = 0;
  for (int k = 0; k < L.K; ++k) {
    sys[k] = PassSys{L.geo_off[k], L.n[k], L.chg_off[k], L.nc[k]};
    n_chg = std::max(n_chg, L.chg_off[k] + L.nc[k]);
  }
  ItemPlan* plan = plan_pass<SourcePolicy, float4, NT, TPT, CH>(s, kPassSource, sys, CH);
  s->grow(s->chgdf, (size_t)2 * n_chg);
  s->grow(s->part64, (size_t)plan->part_len);
  k_pack_chg_df<<<blocks_for(n_chg, 256), 256, 0, s->stream>>>(n_chg, s->chg.p, s->chgdf.p);
  BIPB_LAUNCHED(s);
  SourcePolicy::Args a{s->tgt64.p, s->part64.p};
  launch_items<SourcePolicy, float4, NT, TPT, CH>(s, kTSource, plan, a, s->chgdf.p, nullptr, 0);
  k_reduce_source<<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      s->lay_dev(L), plan->tab.p, s->part64.p, kInv4Pi / m.eps_in, b);
  BIPB_LAUNCHED(s);
}

void reaction_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, double* phi_reac,
                   double* e_out) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  std::vector<PassSys> sys(L.K);
  for (int k = 0; k < L.K; ++k) sys[k] = PassSys{L.chg_off[k], L.nc[k], L.vec_off[k] / 2, L.n[k]};
  ItemPlan* plan = plan_pass<ReactionPolicy, float4, NT, TPT, CH>(s, kPassReaction, sys, CH);
  s->grow(s->recdf, (size_t)2 * L.len);  // 4 float4 per element
  s->grow(s->part64, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  k_pack_df<<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(lay, false, s->tgt64.p, u, s->recdf.p,
                                                                          nullptr, 0);
  BIPB_LAUNCHED(s);
  ReactionPolicy::Args a{s->chg.p, s->part64.p, df_const_impl(s, m)};
  launch_items<ReactionPolicy, float4, NT, TPT, CH>(s, kTReaction, plan, a, s->recdf.p, nullptr, 0);
  k_reduce_reaction<<<L.K, 1024, 0, s->stream>>>(plan->tab.p, lay, s->part64.p, s->chg.p, phi_reac, e_out);
  BIPB_LAUNCHED(s);
}

void potential_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, bool inside,
                    int n_pts, const double4_32a* pts, const double4_32a* pts2, double* out) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  // surface integral: targets are the points (shared by every system), sources the elements
  std::vector<PassSys> sys(L.K);
  for (int k = 0; k < L.K; ++k) sys[k] = PassSys{0, n_pts, L.vec_off[k] / 2, L.n[k]};
  s->grow(s->recdf, (size_t)2 * L.len);  // 4 float4 per element
  const int4* lay = s->lay_dev(L);
  k_pack_df<<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(lay, false, s->tgt64.p, u, s->recdf.p,
                                                                          nullptr, 0);
  BIPB_LAUNCHED(s);
  ReactionPolicy::Args a{pts, nullptr, df_const_impl(s, m)};
  ItemPlan* plan;
  if (inside) {
    plan = plan_pass<ReactionPolicy, float4, NT, TPT, CH>(s, kPassPotIn, sys, CH);
    s->grow(s->part64, (size_t)plan->part_len);
    a.part = s->part64.p;
    launch_items<ReactionPolicy, float4, NT, TPT, CH>(s, kTPotential, plan, a, s->recdf.p, nullptr, 0);
  } else {
    plan = plan_pass<ExteriorPolicy, float4, NT, TPT, CH>(s, kPassPotOut, sys, CH);
    s->grow(s->part64, (size_t)plan->part_len);
    a.part = s->part64.p;
    launch_items<ExteriorPolicy, float4, NT, TPT, CH>(s, kTPotential, plan, a, s->recdf.p, nullptr, 0);
  }
  k_reduce_points<<<dim3(blocks_for(n_pts, 256), L.K), 256, 0, s->stream>>>(plan->tab.p, s->part64.p, n_pts, 1,
                                                                           kInv4Pi, 0, out);
  BIPB_LAUNCHED(s);
  if (!inside) return;
  // S1 at the points (Eq. eq_inside): targets the points with a zero normal, sources the charges
  int n_chg = 0;
  for (int k = 0; k < L.K; ++k) {
    sys[k] = PassSys{0, n_pts, L.chg_off[k], L.nc[k]};
    n_chg = std::max(n_chg, L.chg_off[k] + L.nc[k]);
  }
  if (n_chg == 0) return;
  ItemPlan* sp = plan_pass<SourcePolicy, float4, NT, TPT, CH>(s, kPassPotSrc, sys, CH);
  s->grow(s->chgdf, (size_t)2 * n_chg);
  s->grow(s->part64, (size_t)sp->part_len);
  k_pack_chg_df<<<blocks_for(n_chg, 256), 256, 0, s->stream>>>(n_chg, s->chg.p, s->chgdf.p);
  BIPB_LAUNCHED(s);
  SourcePolicy::Args b{pts2, s->part64.p};
  launch_items<SourcePolicy, float4, NT, TPT, CH>(s, kTPotential, sp, b, s->chgdf.p, nullptr, 0);
  k_reduce_points<<<dim3(blocks_for(n_pts, 256), L.K), 256, 0, s->stream>>>(sp->tab.p, s->part64.p, n_pts, 2,
                                                                           kInv4Pi / m.eps_in, 1, out);
  BIPB_LAUNCHED(s);
}

void coulomb_pass(Surface* s, const SysLayout& L, const int4* tab, double* part, int* blocks) {
  int nc_max = 1;
  for (int k = 0; k < L.K; ++k) nc_max = std::max(nc_max, L.nc[k]);
  *blocks = blocks_for(nc_max, 256);
  k_coulomb<<<dim3(*blocks, L.K), 256, 0, s->stream>>>(tab, s->chg.p, part);
  BIPB_LAUNCHED(s);
}

void energy_row_pass(Surface* s, const SysLayout& L, const bipb_medium& m, double* c) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  std::vector<PassSys> sys(L.K);
  int n_chg = 0;
  for (int k = 0; k < L.K; ++k) {
    sys[k] = PassSys{L.geo_off[k], L.n[k], L.chg_off[k], L.nc[k]};
    n_chg = std::max(n_chg, L.chg_off[k] + L.nc[k]);
  }
  ItemPlan* plan = plan_pass<EnergyRowPolicy, float4, NT, TPT, CH>(s, kPassRow, sys, CH);
  s->grow(s->chgdf, (size_t)2 * n_chg);
  s->grow(s->part64, (size_t)plan->part_len);
  k_pack_chg_df<<<blocks_for(n_chg, 256), 256, 0, s->stream>>>(n_chg, s->chg.p, s->chgdf.p);
  BIPB_LAUNCHED(s);
  EnergyRowPolicy::Args a{s->tgt64.p, s->part64.p, df_const_impl(s, m)};
  launch_items<EnergyRowPolicy, float4, NT, TPT, CH>(s, kTRow, plan, a, s->chgdf.p, nullptr, 0);
  k_energy_row_reduce<<<dim3(blocks_for(2 * L.max_n, 256), L.K), 256, 0, s->stream>>>(
      s->lay_dev(L), plan->tab.p, s->part64.p, s->tgt64.p, c);
  BIPB_LAUNCHED(s);
}

void grad_pass(Surface* s, const SysLayout& L, const bipb_medium& m, const double* u, const double* lam, double* dq,
               double* dy) {
  constexpr int NT = 128, TPT = 1, CH = 32;
  std::vector<PassSys> sys(L.K);
  for (int k = 0; k < L.K; ++k) sys[k] = PassSys{L.chg_off[k], L.nc[k], L.vec_off[k] / 2, L.n[k]};
  ItemPlan* plan = plan_pass<GradPolicy, float4, NT, TPT, CH>(s, kPassGrad, sys, CH);
  s->grow(s->recdf, (size_t)5 * L.len / 2);  // 5 float4 per element
  s->grow(s->part64, (size_t)plan->part_len);
  const int4* lay = s->lay_dev(L);
  k_pack_grad<<<dim3(blocks_for(L.max_n, 256), L.K), 256, 0, s->stream>>>(lay, s->tgt64.p, u, lam, s->recdf.p);
  BIPB_LAUNCHED(s);
  const double inv = 1.0 / m.eps_in;
  const float inv_hi = (float)inv;
  GradPolicy::Args a{s->chg.p, s->part64.p, df_const_impl(s, m), df{inv_hi, (float)(inv - (double)inv_hi)}};
  launch_items<GradPolicy, float4, NT, TPT, CH>(s, kTGrad, plan, a, s->recdf.p, nullptr, 0);
  k_reduce_grad<<<dim3(blocks_for(L.max_nc, 256), L.K), 256, 0, s->stream>>>(plan->tab.p, lay, s->part64.p,
                                                                              s->chg.p, dq, dy);
  BIPB_LAUNCHED(s);
}

}  // namespace bipb
