// Pair passes of the direct-sum pipeline (Sec. 2.4): the mat-vec of Eqs. 5-6
// and its transpose, the source term (Eq. for S1, S2), the reaction potential
// and solvation energy (Eq. for E_sol), and the energy gradient.
//
// Every pass has the same shape: targets in registers (several per thread),
// sources streamed through shared memory in chunks, each CTA covering one
// target tile against one split of the source chunks and writing per-split
// partial sums; a reduction kernel then adds the splits in a fixed order in
// FP64, applies the 1/(4 pi) and the diagonal, and writes the output.  The
// fixed order makes every pass bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr double kInv4Pi = 1.0 / (4.0 * kPi);
constexpr double kFar = 1.0e10;  // position of padding records

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

__device__ __forceinline__ bool skipped(const int* skip) { return skip != nullptr && *skip != 0; }

// ------------------------------------------------------------------ policies
// A policy P describes one pass: the target state loaded into registers, the
// source record (RW vectors of 4), the accumulator and the pair update.

template <typename T>
struct ElemTgt {
  T x, y, z, nx, ny, nz;
};

template <typename T, bool TRANS>
struct MatvecPolicy {
  using V4 = typename V4T<T>::type;
  static constexpr int RW = 2;
  static constexpr bool SELF = true;
  using Tgt = ElemTgt<T>;
  struct Acc {
    T p, q;
  };
  struct Args {
    const V4* tgt;  // 2 per element: (x, y, z, area), (nx, ny, nz, 0)
    const V4* rec;  // RW per source
    T* part;        // [split][2][n]
    int n;
    PairConst<T> c;
  };
  __device__ static void load(const Args& a, int i, Tgt& t) {
    V4 g = a.tgt[2 * i], v = a.tgt[2 * i + 1];
    t = Tgt{g.x, g.y, g.z, v.x, v.y, v.z};
  }
  __device__ static void zero(Acc& acc) { acc.p = T(0), acc.q = T(0); }
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
  __device__ static void store(const Args& a, int split, int i, const Acc& acc) {
    a.part[(size_t)split * 2 * a.n + i] = acc.p;
    a.part[(size_t)split * 2 * a.n + a.n + i] = acc.q;
  }
};

// Source term: target element i, source charge k with record (y_k, q_k), d = x_i - y_k:
//   4 pi eps_in S1 += q s,   4 pi eps_in S2 += -q (n_i.d) s^3   (d/dnu_x = +n_x.grad_x)
struct SourcePolicy {
  static constexpr int RW = 1;
  static constexpr bool SELF = false;
  using Tgt = ElemTgt<double>;
  struct Acc {
    double s1, s2;
  };
  struct Args {
    const double4_32a* geo;
    const double4_32a* nrm;
    const double4_32a* rec;  // (y, q)
    double* part;        // [split][2][n]
    int n;
  };
  __device__ static void load(const Args& a, int i, Tgt& t) {
    double4_32a g = a.geo[i], v = a.nrm[i];
    t = Tgt{g.x, g.y, g.z, v.x, v.y, v.z};
  }
  __device__ static void zero(Acc& acc) { acc.s1 = 0.0, acc.s2 = 0.0; }
  template <bool MASK>
  __device__ static void pair(const Args&, const Tgt& t, const double4_32a* r, bool, Acc& acc) {
    const double4_32a A = r[0];
    double dx = t.x - A.x, dy = t.y - A.y, dz = t.z - A.z;
    double s = fmin(rsqrt(dx * dx + dy * dy + dz * dz), kSMaxD);
    double qs = A.w * s;
    acc.s1 += qs;
    acc.s2 -= qs * (s * s) * (t.nx * dx + t.ny * dy + t.nz * dz);
  }
  __device__ static void store(const Args& a, int split, int i, const Acc& acc) {
    a.part[(size_t)split * 2 * a.n + i] = acc.s1;
    a.part[(size_t)split * 2 * a.n + a.n + i] = acc.s2;
  }
};

struct PointTgt {
  double x, y, z;
};

// Reaction potential at a charge y_k from the surface (forward FP64 record
// (x_j, a_j = ds psi_j), m_j = ds phi_j n_j), d = y_k - x_j:
//   4 pi phi_reac += s [ (1 - e) a_j + (eps t - 1) (m_j.d) s^2 ]  (K1 psi + K2 phi, n_j only)
struct ReactionPolicy {
  static constexpr int RW = 2;
  static constexpr bool SELF = false;
  using Tgt = PointTgt;
  struct Acc {
    double p;
  };
  struct Args {
    const double4_32a* pts;  // (y, q)
    const double4_32a* rec;
    double* part;  // [split][n_pts]
    int n;         // number of charges
    PairConst<double> c;
  };
  __device__ static void load(const Args& a, int k, Tgt& t) {
    double4_32a g = a.pts[k];
    t = Tgt{g.x, g.y, g.z};
  }
  __device__ static void zero(Acc& acc) { acc.p = 0.0; }
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const double4_32a* r, bool, Acc& acc) {
    const double4_32a A = r[0], B = r[1];
    double dx = t.x - A.x, dy = t.y - A.y, dz = t.z - A.z;
    double r2 = dx * dx + dy * dy + dz * dz;
    double s, rr, e;
    radial<false>(r2, false, a.c, s, rr, e);
    double t1 = e * (rr * a.c.kappa) + e;
    double cm = B.x * dx + B.y * dy + B.z * dz;
    double p = A.w - e * A.w;
    p += ((a.c.eps * t1 - 1.0) * cm) * (s * s);
    acc.p += p * s;
  }
  __device__ static void store(const Args& a, int split, int k, const Acc& acc) {
    a.part[(size_t)split * a.n + k] = acc.p;
  }
};

// Energy gradient at charge y_k.  Records per element j: (x_j, a_j),
// (m_j, lphi_j), (p_j = lpsi_j n_j, 0) with u = [phi; psi] and the adjoint
// lam = [lphi; lpsi].  With d = y_k - x_j (times 4 pi):
//   phi_reac  += s [ (1-e) a + (eps t - 1)(m.d) s^2 ]
//   grad_A    += s^3 [ (eps t - 1) m + ((t - 1) a - (eps w - 3)(m.d) s^2) d ]
//   src_B     += s [ lphi + (p.d) s^2 ]
//   grad_B    += s^3 [ p - (lphi + 3 (p.d) s^2) d ]
// grad_A is the y-gradient of the energy row (d/dy of K1(y, x_j) and
// K2(y, x_j)); src_B and grad_B are the adjoint-weighted source column
// (G0(x_j, y) and dG0(x_j, y)/dnu_x) and its y-gradient.
struct GradPolicy {
  static constexpr int RW = 3;
  static constexpr bool SELF = false;
  using Tgt = PointTgt;
  struct Acc {
    double p, sb, ga[3], gb[3];
  };
  struct Args {
    const double4_32a* pts;
    const double4_32a* rec;
    double* part;  // [split][8][n_pts]
    int n;
    PairConst<double> c;
  };
  __device__ static void load(const Args& a, int k, Tgt& t) {
    double4_32a g = a.pts[k];
    t = Tgt{g.x, g.y, g.z};
  }
  __device__ static void zero(Acc& acc) {
    acc.p = acc.sb = 0.0;
    for (int m = 0; m < 3; ++m) acc.ga[m] = acc.gb[m] = 0.0;
  }
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const double4_32a* r, bool, Acc& acc) {
    const double4_32a A = r[0], B = r[1], C = r[2];
    double d[3] = {t.x - A.x, t.y - A.y, t.z - A.z};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double s, rr, e;
    radial<false>(r2, false, a.c, s, rr, e);
    double kr = rr * a.c.kappa;
    double t1 = e * kr + e;
    double w = e * (3.0 + kr * (3.0 + kr));
    double s2 = s * s, s3 = s2 * s;
    double cm = B.x * d[0] + B.y * d[1] + B.z * d[2];
    double cp = C.x * d[0] + C.y * d[1] + C.z * d[2];
    double et1 = a.c.eps * t1 - 1.0;
    acc.p += s * ((A.w - e * A.w) + et1 * cm * s2);
    double fa = (t1 - 1.0) * A.w - (a.c.eps * w - 3.0) * cm * s2;
    double mv[3] = {B.x, B.y, B.z}, pv[3] = {C.x, C.y, C.z};
    double lphi = B.w;
    acc.sb += s * (lphi + cp * s2);
    double fb = lphi + 3.0 * cp * s2;
    for (int m = 0; m < 3; ++m) {
      acc.ga[m] += s3 * (et1 * mv[m] + fa * d[m]);
      acc.gb[m] += s3 * (pv[m] - fb * d[m]);
    }
  }
  __device__ static void store(const Args& a, int split, int k, const Acc& acc) {
    double* o = a.part + (size_t)split * 8 * a.n + k;
    o[0] = acc.p;
    o[(size_t)a.n] = acc.sb;
    for (int m = 0; m < 3; ++m) {
      o[(size_t)(2 + m) * a.n] = acc.ga[m];
      o[(size_t)(5 + m) * a.n] = acc.gb[m];
    }
  }
};

// ------------------------------------------------------------------ tiled driver
// grid = (n_tiles, n_splits).  CTA (x, y) handles targets
// [x*NT*TPT, (x+1)*NT*TPT) (thread t owns x*NT*TPT + k*NT + t, k < TPT)
// against sources [y*ns/S, (y+1)*ns/S) with S = n_splits, staged through
// shared memory CH records at a time (the last chunk of a split may be short).
template <class P, typename V4, int NT, int TPT, int CH>
__global__ void __launch_bounds__(NT) k_tiled(typename P::Args a, int n_targets, int n_sources, int n_splits,
                                              const V4* __restrict__ rec, const int* __restrict__ skip) {
  __shared__ V4 sh[CH * P::RW];
  if (skipped(skip)) return;
  const int t0 = blockIdx.x * NT * TPT;
  typename P::Tgt tg[TPT];
  typename P::Acc acc[TPT];
  int idx[TPT];
#pragma unroll
  for (int k = 0; k < TPT; ++k) {
    idx[k] = t0 + k * NT + threadIdx.x;
    P::load(a, min(idx[k], n_targets - 1), tg[k]);
    P::zero(acc[k]);
  }
  const int s0 = (int)((int64_t)blockIdx.y * n_sources / n_splits);
  const int s1 = (int)((int64_t)(blockIdx.y + 1) * n_sources / n_splits);
  for (int j0 = s0; j0 < s1; j0 += CH) {
    const int cnt = min(CH, s1 - j0);
    __syncthreads();
    const V4* src = rec + (size_t)j0 * P::RW;
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
  }
#pragma unroll
  for (int k = 0; k < TPT; ++k)
    if (idx[k] < n_targets) P::store(a, blockIdx.y, idx[k], acc[k]);
}

// Source split count: every split gets the same number of sources (+-1), and
// the CTA count fills whole waves of resident CTAs (slots = SMs x CTAs per SM)
// as closely as possible, so that no SM idles while others finish a tail.
PassTiling make_tiling(int64_t n_targets, int64_t n_sources, int targets_per_cta, int slots, int min_src) {
  PassTiling t;
  t.n_tiles = (int)((n_targets + targets_per_cta - 1) / targets_per_cta);
  const int max_s = (int)std::max<int64_t>(1, std::min<int64_t>(n_sources / std::max(min_src, 1), 4096));
  auto eff = [&](int sp) {
    const long ctas = (long)t.n_tiles * sp;
    const long waves = (ctas + slots - 1) / slots;
    return (double)ctas / ((double)waves * slots);
  };
  double best = 0.0;
  for (int sp = 1; sp <= max_s; ++sp) best = std::max(best, eff(sp));
  int best_s = 1;
  for (int sp = 1; sp <= max_s; ++sp)
    if (eff(sp) >= 0.98 * best) {  // the fewest splits within 2 % of the best fill
      best_s = sp;
      break;
    }
  t.n_splits = best_s;
  return t;
}

// ------------------------------------------------------------------ pack / reduce
// Forward record of element j from u = [phi; psi]: (x, a = ds psi), (m = ds phi n, 0);
// transposed record from w = [wphi; wpsi]: (x, wphi), (p = wpsi n, 0).
template <typename V4, typename T>
__global__ void k_pack(int n, int n_pad, bool transpose, const double4_32a* __restrict__ geo,
                       const double4_32a* __restrict__ nrm, const double* __restrict__ u, V4* __restrict__ rec,
                       const int* __restrict__ skip) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pad || skipped(skip)) return;
  V4 r0, r1;
  if (j < n) {
    double4_32a g = geo[j], v = nrm[j];
    double phi = u[j], psi = u[n + j];
    double sc = transpose ? phi : g.w * psi;     // 4th slot
    double f = transpose ? psi : g.w * phi;      // multiplies the normal
    r0.x = (T)g.x, r0.y = (T)g.y, r0.z = (T)g.z, r0.w = (T)sc;
    r1.x = (T)(f * v.x), r1.y = (T)(f * v.y), r1.z = (T)(f * v.z), r1.w = (T)0;
  } else {
    r0.x = r0.y = r0.z = (T)kFar, r0.w = (T)0;
    r1.x = r1.y = r1.z = r1.w = (T)0;
  }
  rec[2 * j] = r0;
  rec[2 * j + 1] = r1;
}

// y_i = diag * u_i - (1/(4 pi)) * scale_i * sum_s part[s][i], i < 2n,
// diag = 1/2 (1 + eps) on the phi half and 1/2 (1 + 1/eps) on the psi half;
// scale_i = area of element (i mod n) for the transpose, 1 otherwise.
template <typename PT>
__global__ void k_reduce_matvec(int n, int n_splits, const PT* __restrict__ part,
                                const double* __restrict__ u, double* __restrict__ y, double d_phi,
                                double d_psi, const double4_32a* __restrict__ geo_for_area,
                                const int* __restrict__ skip) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n || skipped(skip)) return;
  double acc = 0.0;
  for (int sp = 0; sp < n_splits; ++sp) acc += (double)part[(size_t)sp * 2 * n + i];
  int e = i < n ? i : i - n;
  double sc = geo_for_area ? geo_for_area[e].w : 1.0;
  y[i] = (i < n ? d_phi : d_psi) * u[i] - kInv4Pi * sc * acc;
}

__global__ void k_reduce_source(int n, int n_splits, const double* __restrict__ part, double scale,
                                double* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  double acc = 0.0;
  for (int sp = 0; sp < n_splits; ++sp) acc += part[(size_t)sp * 2 * n + i];
  b[i] = scale * acc;
}

// phi_reac_k = (1/(4 pi)) sum_s part; E = KCAL/2 sum_k q_k phi_reac_k (one block, fixed order).
__global__ void k_reduce_reaction(int nc, int n_splits, const double* __restrict__ part,
                                  const double4_32a* __restrict__ pts, double* __restrict__ phi_reac,
                                  double* __restrict__ e_out) {
  __shared__ double red[1024];
  double local = 0.0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    double acc = 0.0;
    for (int sp = 0; sp < n_splits; ++sp) acc += part[(size_t)sp * nc + k];
    acc *= kInv4Pi;
    if (phi_reac) phi_reac[k] = acc;
    local += pts[k].w * acc;
  }
  red[threadIdx.x] = local;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && e_out) *e_out = 0.5 * kKcal * red[0];
}

__global__ void k_energy_row_reduce(int n, int n_splits, const double* __restrict__ part,
                                    const double4_32a* __restrict__ geo, double* __restrict__ c) {
  // part[s][0][j] = sum_k q_k 4pi K2(y_k, x_j) with n_j, part[s][1][j] = sum_k q_k 4pi K1(y_k, x_j)
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  double acc = 0.0;
  for (int sp = 0; sp < n_splits; ++sp) acc += part[(size_t)sp * 2 * n + i];
  int e = i < n ? i : i - n;
  c[i] = geo[e].w * kInv4Pi * acc;
}

// Energy row c: target element j, source charge k (record (y_k, q_k)), d = y_k - x_j:
//   4 pi K2(y_k, x_j) = (eps t - 1) (n_j.d) s^3,  4 pi K1(y_k, x_j) = (1 - e) s
struct EnergyRowPolicy {
  static constexpr int RW = 1;
  static constexpr bool SELF = false;
  using Tgt = ElemTgt<double>;
  struct Acc {
    double cphi, cpsi;
  };
  struct Args {
    const double4_32a* geo;
    const double4_32a* nrm;
    double* part;
    int n;
    PairConst<double> c;
  };
  __device__ static void load(const Args& a, int i, Tgt& t) {
    double4_32a g = a.geo[i], v = a.nrm[i];
    t = Tgt{g.x, g.y, g.z, v.x, v.y, v.z};
  }
  __device__ static void zero(Acc& acc) { acc.cphi = 0.0, acc.cpsi = 0.0; }
  template <bool MASK>
  __device__ static void pair(const Args& a, const Tgt& t, const double4_32a* r, bool, Acc& acc) {
    const double4_32a A = r[0];
    double dx = A.x - t.x, dy = A.y - t.y, dz = A.z - t.z;
    double s, rr, e;
    radial<false>(dx * dx + dy * dy + dz * dz, false, a.c, s, rr, e);
    double t1 = e * (rr * a.c.kappa) + e;
    double cj = t.nx * dx + t.ny * dy + t.nz * dz;
    acc.cphi += A.w * (a.c.eps * t1 - 1.0) * cj * (s * s * s);
    acc.cpsi += A.w * (1.0 - e) * s;
  }
  __device__ static void store(const Args& a, int split, int i, const Acc& acc) {
    a.part[(size_t)split * 2 * a.n + i] = acc.cphi;
    a.part[(size_t)split * 2 * a.n + a.n + i] = acc.cpsi;
  }
};

__global__ void k_pack_grad(int n, int n_pad, const double4_32a* __restrict__ geo,
                            const double4_32a* __restrict__ nrm, const double* __restrict__ u,
                            const double* __restrict__ lam, double4_32a* __restrict__ rec) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pad) return;
  double4_32a r0, r1, r2;
  if (j < n) {
    double4_32a g = geo[j], v = nrm[j];
    double aphi = g.w * u[j];
    r0 = make_double4_32a(g.x, g.y, g.z, g.w * u[n + j]);
    r1 = make_double4_32a(aphi * v.x, aphi * v.y, aphi * v.z, lam[j]);
    double lp = lam[n + j];
    r2 = make_double4_32a(lp * v.x, lp * v.y, lp * v.z, 0.0);
  } else {
    r0 = make_double4_32a(kFar, kFar, kFar, 0.0);
    r1 = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    r2 = r1;
  }
  rec[3 * j] = r0;
  rec[3 * j + 1] = r1;
  rec[3 * j + 2] = r2;
}

__global__ void k_reduce_grad(int nc, int n_splits, const double* __restrict__ part,
                              const double4_32a* __restrict__ pts, double inv_eps_in,
                              double* __restrict__ dq, double* __restrict__ dy) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int sp = 0; sp < n_splits; ++sp)
    for (int c = 0; c < 8; ++c) v[c] += part[(size_t)sp * 8 * nc + (size_t)c * nc + k];
  double q = pts[k].w;
  dq[k] = 0.5 * kInv4Pi * (v[0] + inv_eps_in * v[1]);
  for (int m = 0; m < 3; ++m) dy[3 * k + m] = 0.5 * q * kInv4Pi * (v[2 + m] + inv_eps_in * v[5 + m]);
}

template <typename T>
PairConst<T> pair_const(const bipb_medium& m) {
  double eps = m.eps_out / m.eps_in;
  PairConst<T> c;
  c.eps = (T)eps;
  c.inveps = (T)(1.0 / eps);
  c.kappa = (T)m.kappa;
  c.nkl2e = (T)(-m.kappa * 1.4426950408889634);
  return c;
}

int blocks_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

__global__ void k_charge_records(int nc, int nc_pad, const double4_32a* __restrict__ chg,
                                 double4_32a* __restrict__ rec) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc_pad) return;
  rec[k] = k < nc ? chg[k] : make_double4_32a(kFar, kFar, kFar, 0.0);
}

// Resident CTAs per SM of one tiled-kernel instantiation (queried once).
template <class P, typename V4, int NT, int TPT, int CH>
int tiled_occupancy() {
  static int occ = [] {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tiled<P, V4, NT, TPT, CH>, NT, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      o = 1;
    }
    return std::max(o, 1);
  }();
  return occ;
}

template <class P, typename V4, int NT, int TPT, int CH>
PassTiling plan_tiled(Surface* s, int64_t n_targets, int64_t n_sources, int min_src) {
  return make_tiling(n_targets, n_sources, NT * TPT, s->num_sms * tiled_occupancy<P, V4, NT, TPT, CH>(), min_src);
}

// Launch of one tiled pass with a tiling from plan_tiled.
template <class P, typename V4, int NT, int TPT, int CH>
void launch_tiled(Surface* s, int kind, const PassTiling& tl, const typename P::Args& a, int64_t n_targets,
                  int64_t n_sources, const V4* rec, const int* skip) {
  dim3 grid(tl.n_tiles, tl.n_splits);
  TimedLaunch tlaunch(s, kind);
  k_tiled<P, V4, NT, TPT, CH><<<grid, NT, 0, s->stream>>>(a, (int)n_targets, (int)n_sources, tl.n_splits, rec,
                                                          skip);
  BIPB_LAUNCHED(s);
}

// FP32 forward / transpose mat-vec variants (the autotuner picks one).
template <bool TRANS, int NT, int TPT, int CH>
void run_matvec32(Surface* s, const PairConst<float>& c, const double* u, double* y, double dphi,
                  double dpsi, const int* skip) {
  const int n = (int)s->n;
  using P = MatvecPolicy<float, TRANS>;
  PassTiling tl = plan_tiled<P, float4, NT, TPT, CH>(s, n, n, CH);
  const int n_pad = n;
  s->grow(s->rec32, (size_t)2 * n_pad);
  s->grow(s->part32, (size_t)tl.n_splits * 2 * n);
  k_pack<float4, float><<<blocks_for(n_pad, 256), 256, 0, s->stream>>>(
      n, n_pad, TRANS, s->geo64.p, s->nrm64.p, u, s->rec32.p, skip);
  BIPB_LAUNCHED(s);
  typename P::Args a{s->tgt32.p, s->rec32.p, s->part32.p, n, c};
  launch_tiled<P, float4, NT, TPT, CH>(s, TRANS ? kTMv32T : kTMv32, tl, a, n, n, s->rec32.p, skip);
  k_reduce_matvec<float><<<blocks_for(2 * n, 256), 256, 0, s->stream>>>(
      n, tl.n_splits, s->part32.p, u, y, dphi, dpsi, TRANS ? s->geo64.p : nullptr, skip);
  BIPB_LAUNCHED(s);
}

template <bool TRANS>
void run_matvec64(Surface* s, const PairConst<double>& c, const double* u, double* y, double dphi,
                  double dpsi, const int* skip) {
  constexpr int NT = 128, TPT = 2, CH = 64;
  const int n = (int)s->n;
  using P = MatvecPolicy<double, TRANS>;
  PassTiling tl = plan_tiled<P, double4_32a, NT, TPT, CH>(s, n, n, CH);
  const int n_pad = n;
  s->grow(s->rec64, (size_t)2 * n_pad);
  s->grow(s->part64, (size_t)tl.n_splits * 2 * n);
  k_pack<double4_32a, double><<<blocks_for(n_pad, 256), 256, 0, s->stream>>>(
      n, n_pad, TRANS, s->geo64.p, s->nrm64.p, u, s->rec64.p, skip);
  BIPB_LAUNCHED(s);
  typename P::Args a{s->tgt64.p, s->rec64.p, s->part64.p, n, c};
  launch_tiled<P, double4_32a, NT, TPT, CH>(s, TRANS ? kTMv64T : kTMv64, tl, a, n, n, s->rec64.p, skip);
  k_reduce_matvec<double><<<blocks_for(2 * n, 256), 256, 0, s->stream>>>(
      n, tl.n_splits, s->part64.p, u, y, dphi, dpsi, TRANS ? s->geo64.p : nullptr, skip);
  BIPB_LAUNCHED(s);
}

}  // namespace

void matvec(Surface* s, const bipb_medium& m, int precision, bool transpose, const double* u, double* y,
            const int* skip) {
  const double eps = m.eps_out / m.eps_in;
  const double dphi = 0.5 * (1.0 + eps), dpsi = 0.5 * (1.0 + 1.0 / eps);
  if (precision == BIPB_FP64) {
    PairConst<double> c = pair_const<double>(m);
    if (transpose)
      run_matvec64<true>(s, c, u, y, dphi, dpsi, skip);
    else
      run_matvec64<false>(s, c, u, y, dphi, dpsi, skip);
    return;
  }
  PairConst<float> c = pair_const<float>(m);
  switch (s->mv32_variant) {
#define BIPB_MV32(I_, NT_, TPT_, CH_)                                    \
  case I_:                                                               \
    if (transpose)                                                       \
      run_matvec32<true, NT_, TPT_, CH_>(s, c, u, y, dphi, dpsi, skip);  \
    else                                                                 \
      run_matvec32<false, NT_, TPT_, CH_>(s, c, u, y, dphi, dpsi, skip); \
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

namespace {
__global__ void k_fill_test_vector(int len, double* u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) u[i] = 0.5 + 0.25 * sin(0.37 * i) + (i & 7) * 0.01;
}
}  // namespace

int autotune_matvec32(Surface* s, const bipb_medium& m, int reps, double* best_ms) {
  const int len = (int)(2 * s->n);
  DevBuf<double> u, y;
  u.ensure(len);
  y.ensure(len);
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
      matvec(s, m, BIPB_FP32, false, u.p, y.p, nullptr);  // warm-up (and buffer growth)
      BIPB_CUDA(cudaEventRecord(a, s->stream));
      for (int r = 0; r < reps; ++r) matvec(s, m, BIPB_FP32, false, u.p, y.p, nullptr);
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

void source_pass(Surface* s, const bipb_medium& m, int r, double* b) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  const int n = (int)s->n, nc = (int)s->nc;
  PassTiling tl = plan_tiled<SourcePolicy, double4_32a, NT, TPT, CH>(s, n, nc, CH);
  const int nc_pad = nc;
  s->grow(s->rec64, (size_t)nc_pad);
  k_charge_records<<<blocks_for(nc_pad, 256), 256, 0, s->stream>>>(nc, nc_pad, s->chg.p + (size_t)r * nc,
                                                                   s->rec64.p);
  BIPB_LAUNCHED(s);
  s->grow(s->part64, (size_t)tl.n_splits * 2 * n);
  SourcePolicy::Args a{s->geo64.p, s->nrm64.p, s->rec64.p, s->part64.p, n};
  launch_tiled<SourcePolicy, double4_32a, NT, TPT, CH>(s, kTSource, tl, a, n, nc, s->rec64.p, nullptr);
  k_reduce_source<<<blocks_for(2 * n, 256), 256, 0, s->stream>>>(n, tl.n_splits, s->part64.p,
                                                                 kInv4Pi / m.eps_in, b);
  BIPB_LAUNCHED(s);
}

void reaction_pass(Surface* s, const bipb_medium& m, int r, const double* u, double* phi_reac,
                   double* e_out) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  const int n = (int)s->n, nc = (int)s->nc;
  PassTiling tl = plan_tiled<ReactionPolicy, double4_32a, NT, TPT, CH>(s, nc, n, CH);
  const int n_pad = n;
  s->grow(s->rec64, (size_t)2 * n_pad);
  k_pack<double4_32a, double><<<blocks_for(n_pad, 256), 256, 0, s->stream>>>(
      n, n_pad, false, s->geo64.p, s->nrm64.p, u, s->rec64.p, nullptr);
  BIPB_LAUNCHED(s);
  s->grow(s->part64, (size_t)tl.n_splits * nc);
  ReactionPolicy::Args a{s->chg.p + (size_t)r * nc, s->rec64.p, s->part64.p, nc, pair_const<double>(m)};
  launch_tiled<ReactionPolicy, double4_32a, NT, TPT, CH>(s, kTReaction, tl, a, nc, n, s->rec64.p, nullptr);
  k_reduce_reaction<<<1, 1024, 0, s->stream>>>(nc, tl.n_splits, s->part64.p, s->chg.p + (size_t)r * nc,
                                               phi_reac, e_out);
  BIPB_LAUNCHED(s);
}

void energy_row_pass(Surface* s, const bipb_medium& m, int r, double* c) {
  constexpr int NT = 128, TPT = 1, CH = 64;
  const int n = (int)s->n, nc = (int)s->nc;
  PassTiling tl = plan_tiled<EnergyRowPolicy, double4_32a, NT, TPT, CH>(s, n, nc, CH);
  const int nc_pad = nc;
  s->grow(s->rec64, (size_t)nc_pad);
  k_charge_records<<<blocks_for(nc_pad, 256), 256, 0, s->stream>>>(nc, nc_pad, s->chg.p + (size_t)r * nc,
                                                                   s->rec64.p);
  BIPB_LAUNCHED(s);
  s->grow(s->part64, (size_t)tl.n_splits * 2 * n);
  EnergyRowPolicy::Args a{s->geo64.p, s->nrm64.p, s->part64.p, n, pair_const<double>(m)};
  launch_tiled<EnergyRowPolicy, double4_32a, NT, TPT, CH>(s, kTRow, tl, a, n, nc, s->rec64.p, nullptr);
  k_energy_row_reduce<<<blocks_for(2 * n, 256), 256, 0, s->stream>>>(n, tl.n_splits, s->part64.p,
                                                                      s->geo64.p, c);
  BIPB_LAUNCHED(s);
}

void grad_pass(Surface* s, const bipb_medium& m, int r, const double* u, const double* lam, double* dq,
               double* dy) {
  constexpr int NT = 128, TPT = 1, CH = 32;
  const int n = (int)s->n, nc = (int)s->nc;
  PassTiling tl = plan_tiled<GradPolicy, double4_32a, NT, TPT, CH>(s, nc, n, CH);
  const int n_pad = n;
  s->grow(s->rec64, (size_t)3 * n_pad);
  k_pack_grad<<<blocks_for(n_pad, 256), 256, 0, s->stream>>>(n, n_pad, s->geo64.p, s->nrm64.p, u, lam,
                                                             s->rec64.p);
  BIPB_LAUNCHED(s);
  s->grow(s->part64, (size_t)tl.n_splits * 8 * nc);
  GradPolicy::Args a{s->chg.p + (size_t)r * nc, s->rec64.p, s->part64.p, nc, pair_const<double>(m)};
  launch_tiled<GradPolicy, double4_32a, NT, TPT, CH>(s, kTGrad, tl, a, nc, n, s->rec64.p, nullptr);
  k_reduce_grad<<<blocks_for(nc, 256), 256, 0, s->stream>>>(nc, tl.n_splits, s->part64.p,
                                                            s->chg.p + (size_t)r * nc, 1.0 / m.eps_in,
                                                            dq, dy);
  BIPB_LAUNCHED(s);
}

}  // namespace bipb
