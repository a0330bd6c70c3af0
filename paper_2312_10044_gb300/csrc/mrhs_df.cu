// Multi-right-hand-side mat-vec in double-float arithmetic (the refinement
// residual of batched solves).
//
// Y = A U for up to 64 right-hand sides of one surface.  A CTA of 256
// threads covers 64 targets x 4 groups of 16 right-hand sides (warp w: group
// w % 4, targets 32 (w / 4) + lane) against one range of sources, staged 16
// at a time in shared memory together with their 64 right-hand-side values.
// Every thread generates the 2 x 2 kernel block of each pair in df64 (the
// K1..K4 of Sec. 2.2.1 times ds_j, df64.cuh) once and applies it to its 16
// right-hand sides with df64 multiply-adds, so the costly generation is
// shared by 16 right-hand sides instead of repeated for each.  Partial sums
// per source split are written in FP64 and added by the FP64 reduction of
// kernels.cu.
#include <algorithm>

#include "df64.cuh"
#include "internal.cuh"

namespace bipb {

namespace {

constexpr int kNB = 64;     // right-hand sides per launch
constexpr int kGB = 16;     // right-hand sides per thread
constexpr int kTgt = 64;    // targets per CTA
constexpr int kNT = 256;    // threads per CTA
constexpr int kCh = 16;     // sources per shared-memory chunk

// items: {t0, s0, s1, split}; u: system b at (b0 + b) * 2n; part: [b][split][2n]
__global__ void __launch_bounds__(kNT, 1) k_mrhs_df(int n, int nb, int n_splits, const int4* __restrict__ items,
                                                    const double4_32a* __restrict__ tgt64, const double* __restrict__ u,
                                                    double* __restrict__ part, DFConst c) {
  __shared__ float4 srec[kCh][4];        // (x.hi, n.hi), (x.lo, n.lo) split as below
  __shared__ float4 ush[kCh][kNB];       // (phi.hi, phi.lo, psi.hi, psi.lo)
  __shared__ df tab[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp & 3;
  const int tl = 32 * (warp >> 2) + lane;
  const int4 item = items[blockIdx.x];
  const int t0 = item.x, s0 = item.y, s1 = item.z, split = item.w;
  if (tid < 32) tab[tid] = df_from_double(exp2((double)tid / 32.0));
  const int ti = t0 + tl;
  const bool tvalid = ti < n;
  df xi[3], ni[3];
  {
    const double4_32a gi = tgt64[2 * min(ti, n - 1)], vi = tgt64[2 * min(ti, n - 1) + 1];
    xi[0] = df_from_double(gi.x), xi[1] = df_from_double(gi.y), xi[2] = df_from_double(gi.z);
    ni[0] = df_from_double(vi.x), ni[1] = df_from_double(vi.y), ni[2] = df_from_double(vi.z);
  }
  df accp[kGB], accq[kGB];
#pragma unroll
  for (int b = 0; b < kGB; ++b) accp[b] = df{0.f, 0.f}, accq[b] = df{0.f, 0.f};

  for (int j0 = s0; j0 < s1; j0 += kCh) {
    const int cnt = min(kCh, s1 - j0);
    __syncthreads();
    if (tid < cnt) {
      const double4_32a gj = tgt64[2 * (j0 + tid)], vj = tgt64[2 * (j0 + tid) + 1];
      const df x0 = df_from_double(gj.x), x1 = df_from_double(gj.y), x2 = df_from_double(gj.z);
      const df n0 = df_from_double(vj.x), n1 = df_from_double(vj.y), n2 = df_from_double(vj.z);
      const df a = df_from_double(gj.w);
      srec[tid][0] = make_float4(x0.hi, x1.hi, x2.hi, a.hi);
      srec[tid][1] = make_float4(x0.lo, x1.lo, x2.lo, a.lo);
      srec[tid][2] = make_float4(n0.hi, n1.hi, n2.hi, 0.f);
      srec[tid][3] = make_float4(n0.lo, n1.lo, n2.lo, 0.f);
    }
    // right-hand-side values: e = (b * 2 + comp) * cnt + q (q fastest: coalesced reads)
    for (int e = tid; e < kNB * 2 * cnt; e += kNT) {
      const int q = e % cnt, bc = e / cnt, b = bc >> 1, comp = bc & 1;
      const double v = b < nb ? u[(int64_t)b * 2 * n + (int64_t)comp * n + j0 + q] : 0.0;
      const df d = df_from_double(v);
      float* dst = reinterpret_cast<float*>(&ush[q][b]) + 2 * comp;
      dst[0] = d.hi;
      dst[1] = d.lo;
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float4 A = srec[q][0], B = srec[q][1], C = srec[q][2], D = srec[q][3];
      const df xj[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
      const df nj[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
      df k[4];
      df_kernel_block<true>(xi, ni, xj, nj, df{A.w, B.w}, !tvalid || j0 + q == ti, c, tab, k);
#pragma unroll
      for (int b = 0; b < kGB; ++b) {
        const float4 uv = ush[q][kGB * g + b];
        const df up = df{uv.x, uv.y}, uq = df{uv.z, uv.w};
        df_mac(accp[b], k[0], up);
        df_mac(accp[b], k[1], uq);
        df_mac(accq[b], k[2], up);
        df_mac(accq[b], k[3], uq);
      }
    }
#pragma unroll
    for (int b = 0; b < kGB; ++b) {
      accp[b] = fast_two_sum(accp[b].hi, accp[b].lo);
      accq[b] = fast_two_sum(accq[b].hi, accq[b].lo);
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

}  // namespace

void matvec_df_mrhs(Surface* s, const SysLayout& L, const DFConst& c, const double* u, double* y, double dphi,
                    double dpsi, const int* skip, int skip_stride) {
  const int n = L.n[0];
  for (int k = 0; k < L.K; ++k)
    BIPB_REQUIRE(L.geo_off[k] == 0 && L.n[k] == n && L.vec_off[k] == 2 * n * k,
                 "the multi-RHS double-float mat-vec needs right-hand sides of one surface");
  const int tiles = (n + kTgt - 1) / kTgt;
  const int slots = s->num_sms;  // one CTA per SM (register bound)
  int S = 1;
  double best = 0.0;
  for (int sp = 1; sp <= std::min(12, std::max(1, n / (4 * kCh))); ++sp) {
    const long ctas = (long)tiles * sp, waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / ((double)waves * slots);
    if (eff > best * 1.02) best = eff, S = sp;
  }
  const uint64_t key = 0x7e0000000000ull ^ ((uint64_t)n << 8) ^ (uint64_t)S;
  auto it = s->plans.find(key);
  if (it == s->plans.end()) {
    auto p = std::make_unique<ItemPlan>();
    std::vector<int4> items;
    for (int t = 0; t < tiles; ++t)
      for (int sp = 0; sp < S; ++sp)
        items.push_back(make_int4(t * kTgt, (int)((int64_t)sp * n / S), (int)((int64_t)(sp + 1) * n / S), sp));
    p->n_items = (int)items.size();
    p->items.ensure(items.size());
    BIPB_CUDA(cudaMemcpyAsync(p->items.p, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              s->stream));
    BIPB_CUDA(cudaStreamSynchronize(s->stream));
    ++s->alloc_gen;
    it = s->plans.emplace(key, std::move(p)).first;
  }
  ItemPlan* plan = it->second.get();
  s->grow(s->part64, (size_t)std::min(L.K, kNB) * S * 2 * n);
  for (int b0 = 0; b0 < L.K; b0 += kNB) {
    const int nb = std::min(kNB, L.K - b0);
    std::vector<int> go(nb, 0), nn(nb, n), co(nb, 0), nc(nb, 0);
    SysLayout Lb = make_layout(go, nn, co, nc);
    const uint64_t tkey = 0x7f0000000000ull ^ ((uint64_t)n << 16) ^ ((uint64_t)S << 8) ^ (uint64_t)nb;
    auto tt = s->plans.find(tkey);
    if (tt == s->plans.end()) {
      auto p = std::make_unique<ItemPlan>();
      std::vector<int4> tab(nb);
      for (int b = 0; b < nb; ++b) tab[b] = make_int4(n, S, b * S * 2 * n, 0);
      p->tab.ensure(nb);
      BIPB_CUDA(cudaMemcpyAsync(p->tab.p, tab.data(), nb * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
      BIPB_CUDA(cudaStreamSynchronize(s->stream));
      ++s->alloc_gen;
      tt = s->plans.emplace(tkey, std::move(p)).first;
    }
    const double* ub = u + (int64_t)b0 * 2 * n;
    double* yb = y + (int64_t)b0 * 2 * n;
    {
      TimedLaunch tl(s, kTMvDF);
      k_mrhs_df<<<plan->n_items, kNT, 0, s->stream>>>(n, nb, S, plan->items.p, s->tgt64.p, ub, s->part64.p, c);
      BIPB_LAUNCHED(s);
    }
    launch_reduce_matvec64(s, Lb, tt->second->tab.p, s->part64.p, ub, yb, dphi, dpsi,
                           skip ? skip + (int64_t)b0 * skip_stride : nullptr, skip_stride);
  }
}

}  // namespace bipb
