// Multi-right-hand-side mat-vec in double-float arithmetic (the refinement
// residual of batched solves).
//
// Y = A U for up to 64 right-hand sides of one surface.  A CTA covers 32
// targets and G groups of 8 right-hand sides (G = 1, 2, 4 or 8, 32 G
// threads) against one range of sources, staged 16 at a time in shared
// memory with their right-hand-side values.  For every chunk the CTA first
// generates the 2 x 2 kernel block of each (target, source) pair in df64 once
// (the K1..K4 of Sec. 2.2.1 times ds_j, df64.cuh; 16 / G pairs per thread)
// into shared memory; then thread (group g, target t) applies the 16 blocks
// of its target to the group's 8 right-hand sides with df64 multiply-adds.  The costly
// generation is thus shared by all right-hand sides of the CTA, and a pass
// over fewer right-hand sides (a refinement step in which most systems have
// converged) uses fewer groups.  Partial sums per source split are written in
// FP64 and added by the FP64 reduction of kernels.cu.
#include <algorithm>

#include "df64.cuh"
#include "internal.cuh"

namespace bipb {

namespace {

constexpr int kNB = 64;     // right-hand sides per launch (at most)
constexpr int kGB = 8;      // right-hand sides per group (per thread)
constexpr int kTgt = 32;    // targets per CTA
constexpr int kCh = 16;     // sources per shared-memory chunk

// Double-float copies made once per pass, so that the hot loop stages plain
// float4 records and never converts from FP64 (GB300 runs FP64 and its
// conversions at a small fraction of the FP32 rate):
//   geo[4 j .. 4 j + 3] = (x.hi, a.hi), (x.lo, a.lo), (n.hi, 0), (n.lo, 0) of element j
//     (x the centred centroid as a 3-vector, a = ds_j, n the normal);
//   u4[b n + j] = (phi.hi, phi.lo, psi.hi, psi.lo) of right-hand side b (the
//     rhs[b]-th of u when rhs is given), element j.
// blockIdx.y < nb packs right-hand side blockIdx.y, blockIdx.y == nb the geometry.
__global__ void k_pack_mrhs_df(int n, int nb, const double4_32a* __restrict__ tgt64, const double* __restrict__ u,
                               const int* __restrict__ rhs, float4* __restrict__ geo, float4* __restrict__ u4) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int b = blockIdx.y;
  if (b < nb) {
    const double* ub = u + (int64_t)(rhs ? rhs[b] : b) * 2 * n;
    const df p = df_from_double(ub[j]), q = df_from_double(ub[n + j]);
    u4[(int64_t)b * n + j] = make_float4(p.hi, p.lo, q.hi, q.lo);
    return;
  }
  const double4_32a g = tgt64[2 * j], v = tgt64[2 * j + 1];
  const df x0 = df_from_double(g.x), x1 = df_from_double(g.y), x2 = df_from_double(g.z), a = df_from_double(g.w);
  const df n0 = df_from_double(v.x), n1 = df_from_double(v.y), n2 = df_from_double(v.z);
  geo[4 * j] = make_float4(x0.hi, x1.hi, x2.hi, a.hi);
  geo[4 * j + 1] = make_float4(x0.lo, x1.lo, x2.lo, a.lo);
  geo[4 * j + 2] = make_float4(n0.hi, n1.hi, n2.hi, 0.f);
  geo[4 * j + 3] = make_float4(n0.lo, n1.lo, n2.lo, 0.f);
}

// Dynamic shared memory of one CTA with G groups: kernel blocks (hi, lo),
// right-hand-side values, source records, exp table.
template <int G>
constexpr int smem_bytes() {
  return 2 * kCh * kTgt * 16 + kGB * G * kCh * 16 + kCh * 4 * 16 + kExpTab * 8;
}

// items: {t0, s0, s1, split}; geo, u4: the packed records of k_pack_mrhs_df;
// part: [b][split][2n]
template <int G>
__global__ void __launch_bounds__(kTgt * G, 512 / (kTgt * G))
    k_mrhs_df(int n, int nb, int n_splits, const int4* __restrict__ items, const float4* __restrict__ geo,
              const float4* __restrict__ u4, double* __restrict__ part, DFConst c) {
  constexpr int NT = kTgt * G;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* kbh = reinterpret_cast<float4*>(smem);           // [kCh][kTgt]: (K2, K1, K4, K3) ds, hi parts
  float4* kbl = kbh + kCh * kTgt;                           // lo parts
  float4* ush = kbl + kCh * kTgt;                           // [8 G][kCh]: (phi.hi, phi.lo, psi.hi, psi.lo)
  float4* srec = ush + kGB * G * kCh;                       // [kCh][4]: x, n split as below
  df* tab = reinterpret_cast<df*>(srec + kCh * 4);          // 2^(j/1024)
  const int tid = threadIdx.x;
  const int g = tid / kTgt, tl = tid % kTgt;  // MAC phase: group g (warp-uniform), target tl
  const int4 item = items[blockIdx.x];
  const int t0 = item.x, s0 = item.y, s1 = item.z, split = item.w;
  df_load_exp_table(tab, c);
  const int ti = t0 + tl;
  const bool tvalid = ti < n;
  df xi[3], ni[3];
  {
    const int64_t r = 4 * (int64_t)min(ti, n - 1);
    const float4 A = geo[r], B = geo[r + 1], C = geo[r + 2], D = geo[r + 3];
    xi[0] = df{A.x, B.x}, xi[1] = df{A.y, B.y}, xi[2] = df{A.z, B.z};
    ni[0] = df{C.x, D.x}, ni[1] = df{C.y, D.y}, ni[2] = df{C.z, D.z};
  }
  df accp[kGB], accq[kGB];
#pragma unroll
  for (int b = 0; b < kGB; ++b) accp[b] = df{0.f, 0.f}, accq[b] = df{0.f, 0.f};

  for (int j0 = s0; j0 < s1; j0 += kCh) {
    const int cnt = min(kCh, s1 - j0);
    __syncthreads();  // the previous chunk's blocks and values have been used
    for (int e = tid; e < 4 * cnt; e += NT) srec[e] = geo[4 * (int64_t)j0 + e];
    // right-hand-side values, e = b * cnt + q (q fastest: coalesced reads)
    for (int e = tid; e < kGB * G * cnt; e += NT) {
      const int q = e % cnt, b = e / cnt;
      ush[b * kCh + q] = b < nb ? u4[(int64_t)b * n + j0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // kernel blocks of (target tl, source q) for q = g, g + G, ...
    for (int q = g; q < cnt; q += G) {
      const float4 A = srec[4 * q], B = srec[4 * q + 1], C = srec[4 * q + 2], D = srec[4 * q + 3];
      const df xj[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
      const df nj[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
      df k[4];
      df_kernel_block<true>(xi, ni, xj, nj, df{A.w, B.w}, !tvalid || j0 + q == ti, c, tab, k);
      kbh[q * kTgt + tl] = make_float4(k[0].hi, k[1].hi, k[2].hi, k[3].hi);
      kbl[q * kTgt + tl] = make_float4(k[0].lo, k[1].lo, k[2].lo, k[3].lo);
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float4 H = kbh[q * kTgt + tl], Lo = kbl[q * kTgt + tl];
      const df k0 = df{H.x, Lo.x}, k1 = df{H.y, Lo.y}, k2 = df{H.z, Lo.z}, k3 = df{H.w, Lo.w};
#pragma unroll
      for (int b = 0; b < kGB; ++b) {
        const float4 uv = ush[(kGB * g + b) * kCh + q];
        const df up = df{uv.x, uv.y}, uq = df{uv.z, uv.w};
        df_mac(accp[b], k0, up);
        df_mac(accp[b], k1, uq);
        df_mac(accq[b], k2, up);
        df_mac(accq[b], k3, uq);
      }
    }
#pragma unroll
    for (int b = 0; b < kGB; ++b) {
      accp[b] = two_sum(accp[b].hi, accp[b].lo);
      accq[b] = two_sum(accq[b].hi, accq[b].lo);
    }
  }
  if (!tvalid) return;
#pragma unroll
  for (int b = 0; b < kGB; ++b) {
    const int bb = kGB * g + b;
    if (bb >= nb) break;
    double* o = part + ((int64_t)bb * n_splits + split) * 2 * n;
    o[ti] = df_to_double(accp[b]);
    o[n + ti] = df_to_double(accq[b]);
  }
}

template <int G>
int mrhs_df_occupancy() {
  static int occ = [] {
    int o = 0;
    if (cudaFuncSetAttribute(k_mrhs_df<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<G>()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mrhs_df<G>, kTgt * G, smem_bytes<G>()) != cudaSuccess) {
      (void)cudaGetLastError();
      o = 1;
    }
    return std::max(o, 1);
  }();
  return occ;
}

template <int G>
void launch_mrhs_df(Surface* s, const ItemPlan* plan, int n, int nb, int S, const DFConst& c) {
  BIPB_CUDA(cudaFuncSetAttribute(k_mrhs_df<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<G>()));
  k_mrhs_df<G><<<plan->n_items, kTgt * G, smem_bytes<G>(), s->stream>>>(n, nb, S, plan->items.p, s->geodf.p,
                                                                       s->udf.p, s->part64.p, c);
  BIPB_LAUNCHED(s);
}

// Work list of one group count: target tiles x source splits filling whole waves.
ItemPlan* mrhs_df_plan(Surface* s, int n, int G, int slots, int* S_out) {
  const int tiles = (n + kTgt - 1) / kTgt;
  int S = 1;
  double best = 0.0;
  for (int sp = 1; sp <= std::min(12, std::max(1, n / (4 * kCh))); ++sp) {
    const long ctas = (long)tiles * sp, waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / ((double)waves * slots);
    if (eff > best * 1.02) best = eff, S = sp;
  }
  *S_out = S;
  const uint64_t key = 0x7e0000000000ull ^ ((uint64_t)n << 12) ^ ((uint64_t)G << 8) ^ (uint64_t)S;
  auto it = s->plans.find(key);
  if (it == s->plans.end()) {
    auto p = std::make_unique<ItemPlan>();
    std::vector<int4> items;
    for (int t = 0; t < tiles; ++t)
      for (int sp = 0; sp < S; ++sp)
        items.push_back(make_int4(t * kTgt, (int)((int64_t)sp * n / S), (int)((int64_t)(sp + 1) * n / S), sp));
    p->n_items = (int)items.size();
    p->items.ensure(items.size(), s->stream);
    BIPB_CUDA(cudaMemcpyAsync(p->items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    ++s->alloc_gen;
    it = s->plans.emplace(key, std::move(p)).first;
  }
  return it->second.get();
}

}  // namespace

void matvec_df_mrhs(Surface* s, const SysLayout& L, const DFConst& c, const double* u, double* y, double dphi,
                    double dpsi, const int* skip, int skip_stride) {
  const int n = L.n[0];
  for (int k = 0; k < L.K; ++k)
    BIPB_REQUIRE(L.geo_off[k] == 0 && L.n[k] == n && L.vec_off[k] == 2 * n * k,
                 "the multi-RHS double-float mat-vec needs right-hand sides of one surface");
  // right-hand sides to compute: all, or those whose skip flag is clear (the
  // refinement residual of a batch in which some systems have converged)
  std::vector<int> act;
  if (skip != nullptr) {
    std::vector<int> flags((size_t)(L.K - 1) * skip_stride + 1);
    BIPB_CUDA(cudaMemcpyAsync(flags.data(), skip, flags.size() * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    for (int k = 0; k < L.K; ++k)
      if (flags[(size_t)k * skip_stride] == 0) act.push_back(k);
  } else {
    for (int k = 0; k < L.K; ++k) act.push_back(k);
  }
  const int n_act = (int)act.size();
  for (int g0 = 0; g0 < n_act; g0 += kNB) {
    const int nb = std::min(kNB, n_act - g0);
    const int G = nb <= kGB ? 1 : nb <= 2 * kGB ? 2 : nb <= 4 * kGB ? 4 : 8;
    const int slots = s->num_sms * (G == 1   ? mrhs_df_occupancy<1>()
                                    : G == 2 ? mrhs_df_occupancy<2>()
                                    : G == 4 ? mrhs_df_occupancy<4>()
                                             : mrhs_df_occupancy<8>());
    int S = 1;
    ItemPlan* plan = mrhs_df_plan(s, n, G, slots, &S);
    s->grow(s->part64, (size_t)nb * S * 2 * n);
    // reduction layout: right-hand side b of this group at vec_off = act[g0 + b] * 2n of u and y
    SysLayout Lb;
    Lb.K = nb;
    Lb.geo_off.assign(nb, 0);
    Lb.n.assign(nb, n);
    Lb.chg_off.assign(nb, 0);
    Lb.nc.assign(nb, 0);
    Lb.vec_off.resize(nb);
    uint64_t h = 0x6d72687364660000ull ^ (uint64_t)n;
    for (int b = 0; b < nb; ++b) {
      Lb.vec_off[b] = act[g0 + b] * 2 * n;
      h = (h ^ (uint64_t)Lb.vec_off[b]) * 0x100000001b3ull;
    }
    Lb.len = (int64_t)nb * 2 * n;
    Lb.max_n = n;
    Lb.key = h;
    const uint64_t tkey = 0x7f0000000000ull ^ ((uint64_t)n << 16) ^ ((uint64_t)S << 8) ^ (uint64_t)nb;
    auto tt = s->plans.find(tkey);
    if (tt == s->plans.end()) {
      auto p = std::make_unique<ItemPlan>();
      std::vector<int4> tab(nb);
      for (int b = 0; b < nb; ++b) tab[b] = make_int4(n, S, b * S * 2 * n, 0);
      p->tab.ensure(nb, s->stream);
      BIPB_CUDA(cudaMemcpyAsync(p->tab.p, tab.data(), nb * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
      BIPB_CUDA(cudaStreamSynchronize(s->stream));
      ++s->alloc_gen;
      tt = s->plans.emplace(tkey, std::move(p)).first;
    }
    const int* rhs = nullptr;
    const double* ub = u + (int64_t)act[g0] * 2 * n;
    if (act[g0 + nb - 1] - act[g0] != nb - 1) {  // not contiguous: pass the indices
      s->grow(s->rhs_idx, (size_t)nb);
      BIPB_CUDA(cudaMemcpyAsync(s->rhs_idx.p, act.data() + g0, nb * sizeof(int), cudaMemcpyHostToDevice, s->stream));
      BIPB_CUDA(cudaStreamSynchronize(s->stream));
      rhs = s->rhs_idx.p;
      ub = u;
    }
    s->grow(s->geodf, (size_t)4 * n);
    s->grow(s->udf, (size_t)nb * n);
    k_pack_mrhs_df<<<dim3((n + 255) / 256, nb + 1), 256, 0, s->stream>>>(n, nb, s->tgt64.p, ub, rhs, s->geodf.p,
                                                                          s->udf.p);
    BIPB_LAUNCHED(s);
    {
      TimedLaunch tl(s, kTMvDF);
      if (G == 1)
        launch_mrhs_df<1>(s, plan, n, nb, S, c);
      else if (G == 2)
        launch_mrhs_df<2>(s, plan, n, nb, S, c);
      else if (G == 4)
        launch_mrhs_df<4>(s, plan, n, nb, S, c);
      else
        launch_mrhs_df<8>(s, plan, n, nb, S, c);
    }
    launch_reduce_matvec64(s, Lb, tt->second->tab.p, s->part64.p, u, y, dphi, dpsi, nullptr, 0);
  }
}

}  // namespace bipb
