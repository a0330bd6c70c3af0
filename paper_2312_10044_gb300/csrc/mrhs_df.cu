// Multi-right-hand-side mat-vec in double-float arithmetic (the refinement
// residual of batched solves), in two forms: df64 multiply-adds on the CUDA
// cores (below; A U for fewer than 16 right-hand sides) and exact digit
// products on the tensor cores (namespace tcx further down; A U for 16 or
// more right-hand sides, and A^T U).
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

#include <cuda_fp16.h>

#include "df64.cuh"
#include "internal.cuh"
#include "tcgen05.cuh"

namespace bipb {

namespace {

constexpr int kNB = 64;     // right-hand sides per launch (at most)
constexpr int kGB = 8;      // right-hand sides per group (per thread)
constexpr int kTgt = 32;    // targets per CTA
constexpr int kCh = 16;     // sources per shared-memory chunk
constexpr int kTcxMinRHS = 16;  // the exact tensor-core form from this many right-hand sides on

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


// ------------------------------------------------------------------ exact tensor-core form
// The same product with the multiply-adds on the tensor cores, exactly.  Row
// i (the phi or psi row of a target) is scaled by 2^e(i) and right-hand side
// b by 2^f(b) so that every value lies below 64 in magnitude; each df64
// kernel value a and each right-hand-side value u is then written as seven
// signed base-128 digits,
//     a = sum_k d_k 128^-k,   u = sum_l t_l 128^-l,   |d_k|, |t_l| <= 68,
// which FP16 holds exactly.  A kind::f16 MMA of digit planes multiplies
// integers exactly and its FP32 accumulator adds them exactly while every
// sum stays below 2^24 (checked on GB300 by a probe), so level L = k + l of
// the product, sum_{k+l=L} d_k t_l, is accumulated without rounding in its
// own 64 TMEM columns (one per right-hand side): per K chunk of 8 sources,
// MMAs A_k [T_0 | .. | T_{6-k}] (N = 64 (7 - k), cut into pieces of at most
// 256) write levels k .. 6.  Levels above 6 (below 2^-46 of the largest
// product) are dropped.  Every 32 K chunks (512 K, which bounds the sums by
// 512 x 7 x 68 x 64 < 2^24) the generating threads read the levels back and
// add sum_L v_L 128^-L to df64 accumulators.
//
// The M = 128 rows of the MMA are the phi rows (0..63) and the psi rows
// (64..127) of 64 targets, so that the seven levels of all 64 right-hand
// sides fit tensor memory (448 of its 512 columns): every df64 kernel block
// is generated once for all 64 right-hand sides, and the multiply-adds cost
// nothing on the CUDA cores.  A^T U is the same pass over the transposed
// blocks (df_kernel_block<.., true>, area 1), with its own row scales and the
// output element's area applied to the FP64 sums.
namespace tcx {

constexpr int kRHS = 64;                        // right-hand sides per CTA (all of a launch)
constexpr int kLv = 7;                          // digits per value = accumulation levels
constexpr int kTgt = 64;                        // targets per CTA: rows t (phi) and 64 + t (psi)
constexpr int kStep = 16;                       // sources per step: two K chunks
constexpr int kKC = 16;                         // K of one chunk (8 sources x phi, psi; one kind::f16 MMA)
constexpr int kChunks = kStep * 2 / kKC;        // K chunks per step
constexpr int kPlane = 128 * kKC * 2;           // one digit plane of one K chunk: 4 KB
constexpr int kAStage = kChunks * kLv * kPlane; // A of one step: 56 KB
constexpr int kBRows = kLv * kRHS;              // 448 rows: digit plane l of U in rows 64 l ..
constexpr int kBChunk = kBRows * kKC * 2;       // 14 KB per K chunk
constexpr int kBBytes = kChunks * kBChunk;      // 28 KB per step
constexpr int kSRec = kStep * 64;               // source records of one step: 1 KB
constexpr int kRing = 3;                        // B and source buffers (step it in buffer it % 3)
constexpr int kGroupChunks = 32;                // K chunks per exact accumulation group (K = 512)
constexpr int kGroup = kGroupChunks / kChunks;  // steps per group
constexpr int kMaxN = 256;                      // largest N of one MMA
constexpr int kOffA = 0;                        // two A stages
constexpr int kOffB = kOffA + 2 * kAStage;
constexpr int kOffS = kOffB + kRing * kBBytes;
constexpr int kOffTab = kOffS + kRing * kSRec;
constexpr int kOffF = kOffTab + kExpTab * 8;    // 2^-f(b) of the right-hand sides
constexpr int kOffBar = kOffF + kRHS * 4;
constexpr int kNumBars = 3 * kRing + 2 * 2 + 2;
constexpr int kSmemBytes = kOffBar + kNumBars * 8 + 16;
constexpr int kGenThreads = 512;
constexpr int kMmaWarp = kGenThreads / 32;      // warp 16: issues the MMAs
constexpr int kLoadWarp = kMmaWarp + 1;         // warp 17: issues the bulk copies
constexpr int kThreads = kGenThreads + 64;
constexpr uint32_t kTmemCols = 512;             // level L at columns 64 L
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 100000000ull;  // per wait while draining after a time-out
static_assert(kChunks == 2 && kGroup * kChunks == kGroupChunks, "steps of two K chunks");
static_assert(kGenThreads == kTgt * kStep / 2, "one thread per (target, source pair) of a step");
static_assert(kOffB % 1024 == 0 && kBChunk % 16 == 0 && kSRec % 16 == 0, "bulk-copy alignment");
static_assert(kOffBar % 8 == 0 && kOffTab % 16 == 0, "alignment");
static_assert(kSmemBytes <= 227 * 1024, "shared memory");
static_assert(kLv * kRHS <= (int)kTmemCols, "levels fit tensor memory");

// byte offset of element (row, k) of a K-major, no-swizzle FP16 tile with K = 16
__host__ __device__ __forceinline__ uint32_t koff(int row, int k) {
  return (uint32_t)((((row >> 3) * 2 + (k >> 3)) * 8 + (row & 7)) * 16 + (k & 7) * 2);
}
// 2^k in FP32 (|k| <= 126) and FP64 (|k| <= 1022)
__device__ __forceinline__ float p2f(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }
__device__ __forceinline__ double p2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }
// the exponent that brings a largest magnitude with floor(log2) lg below 64 (2^5 <= m 2^e < 2^6),
// clamped to [-100, 100]; 0 for zero
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  const int lg = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;
  return max(-100, min(100, 5 - lg));
}

// a (df64, |a| below 64 up to rounding) as seven base-128 digits, exactly
// up to 2^-43: a = sum_k d[k] 128^-k + rest.  The leading part gives three
// digits by exact FP32 steps; the trailing part (at most 2^-19) joins at the
// fourth, which may then reach 68 in magnitude.
__device__ __forceinline__ void digits7(df a, float* d) {
  float r = a.hi;
  d[0] = rintf(r);
  r = __fsub_rn(r, d[0]);
  d[1] = rintf(__fmul_rn(r, 128.f));
  r = __fsub_rn(__fmul_rn(r, 128.f), d[1]);
  d[2] = rintf(__fmul_rn(r, 128.f));
  r = __fsub_rn(__fmul_rn(r, 128.f), d[2]);
  const df t = two_sum(__fmul_rn(r, 128.f), __fmul_rn(a.lo, 2097152.f));  // units 128^-3
  d[3] = rintf(t.hi);
  r = __fadd_rn(__fsub_rn(t.hi, d[3]), t.lo);
  d[4] = rintf(__fmul_rn(r, 128.f));
  r = __fsub_rn(__fmul_rn(r, 128.f), d[4]);
  d[5] = rintf(__fmul_rn(r, 128.f));
  r = __fsub_rn(__fmul_rn(r, 128.f), d[5]);
  d[6] = rintf(__fmul_rn(r, 128.f));
}

// Row scale exponents: for target i the largest |K2 ds|, |K1 ds| (phi row)
// and |K4 ds|, |K3 ds| (psi row) over all sources j != i, in df64 (the same
// values the kernel digitises).  One thread per target.
template <bool TRANS>
__global__ void __launch_bounds__(128) k_tcx_rowexp(int n, const float4* __restrict__ geo, DFConst c,
                                                    int2* __restrict__ rowexp) {
  __shared__ float4 sh[4 * 64];
  __shared__ __align__(16) df tab[kExpTab];
  df_load_exp_table(tab, c);
  const int i = blockIdx.x * 128 + threadIdx.x;
  const int ii = min(i, n - 1);
  df xi[3], ni[3];
  {
    const float4 A = geo[4 * (size_t)ii], B = geo[4 * (size_t)ii + 1], C = geo[4 * (size_t)ii + 2],
                 D = geo[4 * (size_t)ii + 3];
    xi[0] = df{A.x, B.x}, xi[1] = df{A.y, B.y}, xi[2] = df{A.z, B.z};
    ni[0] = df{C.x, D.x}, ni[1] = df{C.y, D.y}, ni[2] = df{C.z, D.z};
  }
  float m0 = 0.f, m1 = 0.f;
  for (int j0 = 0; j0 < n; j0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * 64; e += 128) sh[e] = geo[4 * (size_t)min(j0 + e / 4, n - 1) + e % 4];
    __syncthreads();
    const int cnt = min(64, n - j0);
    for (int q = 0; q < cnt; ++q) {
      const float4 A = sh[4 * q], B = sh[4 * q + 1], C = sh[4 * q + 2], D = sh[4 * q + 3];
      const df xj[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
      const df nj[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
      df k[4];
      df_kernel_block<true, TRANS>(xi, ni, xj, nj, TRANS ? df{1.f, 0.f} : df{A.w, B.w}, j0 + q == ii, c, tab, k);
      m0 = fmaxf(m0, fmaxf(fabsf(k[0].hi), fabsf(k[1].hi)));
      m1 = fmaxf(m1, fmaxf(fabsf(k[2].hi), fabsf(k[3].hi)));
    }
  }
  if (i < n) rowexp[i] = make_int2(scale_exp(m0), scale_exp(m1));
}

// colmax[b] = max |u_b| over the 2n values (FP32 bits; colmax zeroed before): grid (x, nb)
__global__ void k_tcx_colmax(int n, const double* __restrict__ u, const int* __restrict__ rhs,
                             unsigned* __restrict__ colmax) {
  const int b = blockIdx.y;
  const double* ub = u + (int64_t)(rhs ? rhs[b] : b) * 2 * n;
  float m = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)ub[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + b, __float_as_uint(m));
}

// U digit tiles: for step x and K chunk kc, row 64 l + b holds digit l of
// u_b 2^f(b), K = 2 j' + c (phi_j, psi_j of the chunk's sources), K-major.
// One thread per (x, kc, b, k).
__global__ void k_tcx_pack_u(int n, int nb, int n_steps, const double* __restrict__ u, const int* __restrict__ rhs,
                             const unsigned* __restrict__ colmax, __half* __restrict__ upk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_steps * kChunks * kRHS * kKC) return;
  const int k = (int)(e % kKC), b = (int)((e / kKC) % kRHS);
  const int kc = (int)((e / (kKC * kRHS)) % kChunks);
  const int64_t x = e / ((int64_t)kKC * kRHS * kChunks);
  const int j = (int)(x * kStep) + kc * (kKC / 2) + (k >> 1), c = k & 1;
  double v = 0.0;
  if (b < nb && j < n)
    v = u[(int64_t)(rhs ? rhs[b] : b) * 2 * n + (int64_t)c * n + j] * p2d(scale_exp(__uint_as_float(colmax[b])));
  unsigned char* tile = reinterpret_cast<unsigned char*>(upk) + x * (int64_t)kBBytes + kc * kBChunk;
#pragma unroll
  for (int l = 0; l < kLv; ++l) {
    const double d = rint(v);
    *reinterpret_cast<__half*>(tile + koff(kRHS * l + b, k)) = __float2half_rn((float)d);
    v = (v - d) * 128.0;
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// This thread's source pair of a step (records Sq, first index jq) against
// target tg: the df64 block, scaled per row, as digit planes written into
// the K chunk's planes at `a` (digit k at a + k kPlane; byte offsets offp and
// offq of the target's phi and psi rows at the pair's K columns).
template <bool EDGE, bool TRANS>
__device__ __forceinline__ void tcx_gen(const df* xi, const df* ni, const float4* Sq, int jq, int tg, int n,
                                        bool tvalid, const DFConst& c, const df* tab, float r0, float r1,
                                        unsigned char* a, uint32_t offp, uint32_t offq) {
  float dg[2][4][kLv];  // [source][value: K2, K1, K4, K3][digit]
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const float4 A = Sq[4 * u], B = Sq[4 * u + 1], C = Sq[4 * u + 2], D = Sq[4 * u + 3];
    const df xj[3] = {df{A.x, B.x}, df{A.y, B.y}, df{A.z, B.z}};
    const df nj[3] = {df{C.x, D.x}, df{C.y, D.y}, df{C.z, D.z}};
    const bool z = EDGE && (!tvalid || jq + u >= n || jq + u == tg);
    df k[4];
    df_kernel_block<EDGE, TRANS>(xi, ni, xj, nj, TRANS ? df{1.f, 0.f} : df{A.w, B.w}, z, c, tab, k);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      df w = df_scale(k[v], v < 2 ? r0 : r1);
      if (EDGE && z) w = df{0.f, 0.f};
      digits7(w, dg[u][v]);
    }
  }
  // phi row: (K2, K1) of sources 0, 1 in the pair's four K columns; psi row: (K4, K3)
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int k = 0; k < kLv; ++k) {
      const __half2 p0 = __floats2half2_rn(dg[0][2 * m][k], dg[0][2 * m + 1][k]);
      const __half2 p1 = __floats2half2_rn(dg[1][2 * m][k], dg[1][2 * m + 1][k]);
      uint2 w;
      w.x = *reinterpret_cast<const uint32_t*>(&p0);
      w.y = *reinterpret_cast<const uint32_t*>(&p1);
      *reinterpret_cast<uint2*>(a + k * kPlane + (m ? offq : offp)) = w;
    }
}

// items: {t0, first step, end step, split}; part: [b][split][2n] for the nb
// right-hand sides of this pass.
template <bool TRANS>
__global__ void __launch_bounds__(kThreads, 1)
    k_mrhs_tcx(int n, int nb, int n_splits, const int4* __restrict__ items, const float4* __restrict__ geo,
               const int2* __restrict__ rowexp, const unsigned* __restrict__ colmax, const __half* __restrict__ upk,
               double* __restrict__ part, DFConst c, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* ufull = reinterpret_cast<uint64_t*>(smem + kOffBar);  // kRing: U digit tiles landed
  uint64_t* sfull = ufull + kRing;                                 // kRing: source records landed
  uint64_t* bfree = sfull + kRing;                                 // kRing: MMAs of the buffer's step finished
  uint64_t* ready = bfree + kRing;                                 // 2: A stage written (16 warp arrivals)
  uint64_t* afree = ready + 2;                                     // 2: MMAs of an A stage finished
  uint64_t* done = afree + 2;                                      // MMAs of a group finished
  uint64_t* drained = done + 1;                                    // levels read back (16 warp arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);
  df* tab = reinterpret_cast<df*>(smem + kOffTab);
  float* finv = reinterpret_cast<float*>(smem + kOffF);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 item = items[blockIdx.x];
  const int t0 = item.x, x0 = item.y, x1 = item.z, split = item.w;
  if (tid == 0) {
    for (int q = 0; q < kRing; ++q) {
      tc::mbar_init(&ufull[q], 1);
      tc::mbar_init(&sfull[q], 1);
      tc::mbar_init(&bfree[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&ready[q], kGenThreads / 32);
      tc::mbar_init(&afree[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drained, kGenThreads / 32);
    tc::fence_mbar_init();
  }
  if (tid < kRHS) finv[tid] = tid < nb ? p2f(-scale_exp(__uint_as_float(colmax[tid]))) : 0.f;
  df_load_exp_table(tab, c);
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int n_it = x1 - x0;
  const int n_groups = (n_it + kGroup - 1) / kGroup;
  bool ok = true;
  int issued = 0, mma_last = -1;  // steps whose copies / MMAs this CTA has issued
  const int wq = warp & 3;
  if (warp == kLoadWarp) {
    if (lane == 0) {
      for (int x = 0; x < n_it; ++x) {
        const int q = x % kRing;
        if (x >= kRing) ok = ok && tc::mbar_wait_timed(&bfree[q], ((x - kRing) / kRing) & 1, kWaitLimitNs);
        if (!ok) break;
        const int st = x0 + x;
        const int cnt = min(kStep, n - st * kStep);
        arrive_expect_tx(&sfull[q], cnt * 64);
        bulk_load(smem + kOffS + q * kSRec, geo + 4 * (int64_t)st * kStep, cnt * 64, &sfull[q]);
        arrive_expect_tx(&ufull[q], kBBytes);
        bulk_load(smem + kOffB + q * kBBytes, reinterpret_cast<const unsigned char*>(upk) + (int64_t)st * kBBytes,
                  kBBytes, &ufull[q]);
        issued = x + 1;
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      for (int it = 0; it < n_it && ok; ++it) {
        const int g = it / kGroup, s = it & 1, q = it % kRing;
        const bool first = it % kGroup == 0, last = it % kGroup == kGroup - 1 || it == n_it - 1;
        if (first && g >= 1) ok = ok && tc::mbar_wait_timed(drained, (g - 1) & 1, kWaitLimitNs);
        ok = ok && tc::mbar_wait_timed(&ready[s], (it >> 1) & 1, kWaitLimitNs);
        ok = ok && tc::mbar_wait_timed(&ufull[q], (it / kRing) & 1, kWaitLimitNs);
        if (!ok) break;
        tc::fence_after_sync();
#pragma unroll
        for (int kc = 0; kc < kChunks; ++kc) {
          const uint32_t bbase = tc::smem_u32(smem + kOffB + q * kBBytes + kc * kBChunk);
#pragma unroll
          for (int k = 0; k < kLv; ++k) {
            const uint64_t da =
                tc::smem_desc(tc::smem_u32(smem + kOffA + s * kAStage + (kc * kLv + k) * kPlane), 128, 256);
            // digit k of A against digit planes 0 .. 6 - k of U (rows 0 .. 64 (7 - k) - 1): levels k .. 6,
            // in pieces of at most 256 rows (8-row groups 256 bytes apart)
#pragma unroll
            for (int n0 = 0; n0 < kRHS * (kLv - k); n0 += kMaxN) {
              const int nn = min(kMaxN, kRHS * (kLv - k) - n0);
              const uint64_t db = tc::smem_desc(bbase + (uint32_t)(n0 / 8) * 256u, 128, 256);
              tc::mma_f16_ss(tmem + kRHS * k + n0, da, db, tc::idesc_f16(128, nn),
                             (k > 0 || kc > 0 || !first) ? 1u : 0u);
            }
          }
        }
        tc::mma_commit(&afree[s]);
        tc::mma_commit(&bfree[q]);
        if (last) tc::mma_commit(done);
        mma_last = it;
      }
    }
    __syncwarp();
  } else {
    // generating warps.  Generation: warp w covers targets 8 (w & 7) + (lane
    // & 7) and source pair sp = 4 (w >> 3) + (lane >> 3) of every step (K
    // chunk sp >> 2, K columns 4 (sp & 3) .. + 3), so that each half-warp's
    // 8-byte digit stores fill 128 contiguous bytes (no bank conflict).
    // Read-back: the thread of TMEM lane r = 32 wq + lane owns row r (the
    // phi row of target r for r < 64, the psi row of target r - 64 after)
    // for right-hand sides 16 (w >> 2) .. + 15.
    const int tr = 8 * (warp & 7) + (lane & 7), sp = 4 * (warp >> 3) + (lane >> 3);
    const int tg = t0 + tr;  // the generated target
    const bool gvalid = tg < n;
    df xi[3], ni[3];
    {
      const int64_t r = 4 * (int64_t)min(tg, n - 1);
      const float4 A = geo[r], B = geo[r + 1], C = geo[r + 2], D = geo[r + 3];
      xi[0] = df{A.x, B.x}, xi[1] = df{A.y, B.y}, xi[2] = df{A.z, B.z};
      ni[0] = df{C.x, D.x}, ni[1] = df{C.y, D.y}, ni[2] = df{C.z, D.z};
    }
    const int2 rg_e = rowexp[min(tg, n - 1)];
    const float r0 = p2f(rg_e.x), r1 = p2f(rg_e.y);
    const uint32_t offp = koff(tr, 4 * (sp & 3)), offq = koff(kTgt + tr, 4 * (sp & 3));
    const int rr = 32 * wq + lane;                      // the read-back row
    const int ti = t0 + (rr & (kTgt - 1));              // its target
    const bool tvalid = ti < n;
    const int cb = warp >> 2;                           // its right-hand sides 16 cb .. 16 cb + 15
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    const uint32_t dthr = tmem + lane_base + 16 * cb;
    const bool tile_edge = t0 + kTgt > n;
    df acc[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) acc[b] = df{0.f, 0.f};
    auto read_back = [&]() {  // acc += sum_L level L 128^-L, exact levels, df64 sums
#pragma unroll
      for (int L = 0; L < kLv; ++L) {
        uint32_t v[16];
        tc::tmem_ld16_async(dthr + kRHS * L, v);
        tc::tmem_wait_ld16(v);
        const float sc = p2f(-7 * L);
#pragma unroll
        for (int b = 0; b < 16; ++b) acc[b] = df_add_f(acc[b], __fmul_rn(__uint_as_float(v[b]), sc));
      }
    };
    auto drain = [&](int d) {
      ok = ok && tc::mbar_wait_timed(done, d & 1, kWaitLimitNs);
      if (!ok) return;
      tc::fence_after_sync();
      read_back();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
    };
    int drained_groups = 0;
    for (int it = 0; it < n_it; ++it) {
      const int s = it & 1, q = it % kRing;
      ok = ok && tc::mbar_wait_timed(&sfull[q], (it / kRing) & 1, kWaitLimitNs);
      if (it >= 2) ok = ok && tc::mbar_wait_timed(&afree[s], ((it - 2) >> 1) & 1, kWaitLimitNs);
      const int d = (it % kGroup == 1 && it > kGroup) ? it / kGroup - 1 : -1;
      if (d >= 0) ok = ok && tc::mbar_wait_timed(done, d & 1, kWaitLimitNs);
      if (!ok) break;
      if (it >= 2) tc::fence_after_sync();
      if (d >= 0) {
        read_back();
        drained_groups = d + 1;
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(drained);
      }
      const int j0 = (x0 + it) * kStep;
      const bool edge = tile_edge || (j0 + kStep > n) || (j0 < t0 + kTgt && j0 + kStep > t0);
      const float4* Sq = reinterpret_cast<const float4*>(smem + kOffS + q * kSRec) + 4 * 2 * sp;
      unsigned char* a = smem + kOffA + s * kAStage + (sp >> 2) * kLv * kPlane;
      if (edge)
        tcx_gen<true, TRANS>(xi, ni, Sq, j0 + 2 * sp, tg, n, gvalid, c, tab, r0, r1, a, offp, offq);
      else
        tcx_gen<false, TRANS>(xi, ni, Sq, j0 + 2 * sp, tg, n, gvalid, c, tab, r0, r1, a, offp, offq);
      tc::fence_proxy_async_smem();  // the generic stores, before the tensor core reads them
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
    }
    for (int d = drained_groups; ok && d < n_groups; ++d) drain(d);
    // unscale by 2^-(e + f) and write this split's partial sums (those of
    // A^T times the output element's area)
    if (ok && tvalid && n_it > 0) {
      const int comp = rr / kTgt;
      const int2 re = rowexp[ti];
      const int e = comp ? re.y : re.x;
      const double area = TRANS ? (double)geo[4 * (int64_t)ti].w + (double)geo[4 * (int64_t)ti + 1].w : 1.0;
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        const int bg = 16 * cb + b;
        if (bg < nb) {
          const df w = df_scale(df_scale(acc[b], p2f(-e)), finv[bg]);
          part[((int64_t)bg * n_splits + split) * 2 * n + (int64_t)comp * n + ti] = df_to_double(w) * area;
        }
      }
    }
  }
  const bool all_ok = __syncthreads_and(ok) != 0;
  if (!all_ok) {
    if (tid == 0) atomicExch(err, 1);
    // a wait ran out: the copies and MMAs this CTA issued land before its
    // shared and tensor memory are given up (each wait bounded again)
    if (warp == kLoadWarp && lane == 0)
      for (int x = max(0, issued - kRing); x < issued; ++x) {
        tc::mbar_wait_timed(&sfull[x % kRing], (x / kRing) & 1, kDrainLimitNs);
        tc::mbar_wait_timed(&ufull[x % kRing], (x / kRing) & 1, kDrainLimitNs);
      }
    if (warp == kMmaWarp && lane == 0 && mma_last >= 0)
      tc::mbar_wait_timed(&bfree[mma_last % kRing], (mma_last / kRing) & 1, kDrainLimitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tcx

// Work list of the exact tensor-core pass: target tiles of 64 x source
// splits (whole steps) filling whole waves of one CTA per SM.
ItemPlan* tcx_plan(Surface* s, int n, int* S_out) {
  const int n_steps = (n + tcx::kStep - 1) / tcx::kStep;
  const int tiles = (n + tcx::kTgt - 1) / tcx::kTgt;
  const int slots = s->num_sms;
  int S = 1;
  double best = 0.0;
  for (int sp = 1; sp <= std::min(16, std::max(1, n_steps / tcx::kGroup)); ++sp) {
    const long ctas = (long)tiles * sp, waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / ((double)waves * slots);
    if (eff > best * 1.02) best = eff, S = sp;
  }
  *S_out = S;
  const uint64_t key = 0x7b0000000000ull ^ ((uint64_t)n << 12) ^ (uint64_t)S;
  auto it = s->plans.find(key);
  if (it == s->plans.end()) {
    auto p = std::make_unique<ItemPlan>();
    std::vector<int4> items;
    for (int t = 0; t < tiles; ++t)
      for (int sp = 0; sp < S; ++sp)
        items.push_back(make_int4(t * tcx::kTgt, (int)((int64_t)sp * n_steps / S),
                                  (int)((int64_t)(sp + 1) * n_steps / S), sp));
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

// The exact tensor-core pass for nb <= 64 right-hand sides (u at ub, or the
// rows rhs[b] of u when rhs is given): row exponents (cached per surface and
// medium), right-hand-side digits, the kernel; writes part64 [b][split][2n]
// and returns the number of splits.
int launch_tcx(Surface* s, int n, int nb, bool transpose, const double* ub, const int* rhs, const DFConst& c) {
  const int dir = transpose ? 1 : 0;
  const int n_steps = (n + tcx::kStep - 1) / tcx::kStep;
  s->grow(s->geodf, (size_t)4 * n);
  k_pack_mrhs_df<<<dim3((n + 255) / 256, 1), 256, 0, s->stream>>>(n, 0, s->tgt64.p, ub, rhs, s->geodf.p, s->udf.p);
  BIPB_LAUNCHED(s);
  const uint64_t gen0 = s->alloc_gen;
  s->grow(s->tcx_rowexp[dir], (size_t)n);
  int2* rowexp = s->tcx_rowexp[dir].p;
  float* key = s->tcx_key[dir];
  if (s->alloc_gen != gen0 || s->tcx_n[dir] != n || key[0] != c.eps.hi || key[1] != c.eps.lo ||
      key[2] != c.kappa.hi || key[3] != c.kappa.lo) {
    if (transpose)
      tcx::k_tcx_rowexp<true><<<(n + 127) / 128, 128, 0, s->stream>>>(n, s->geodf.p, c, rowexp);
    else
      tcx::k_tcx_rowexp<false><<<(n + 127) / 128, 128, 0, s->stream>>>(n, s->geodf.p, c, rowexp);
    BIPB_LAUNCHED(s);
    s->tcx_n[dir] = n;
    key[0] = c.eps.hi, key[1] = c.eps.lo, key[2] = c.kappa.hi, key[3] = c.kappa.lo;
  }
  s->grow(s->tcx_colmax, (size_t)kNB);
  BIPB_CUDA(cudaMemsetAsync(s->tcx_colmax.p, 0, kNB * sizeof(unsigned), s->stream));
  tcx::k_tcx_colmax<<<dim3((unsigned)std::min(64, (2 * n + 255) / 256), nb), 256, 0, s->stream>>>(n, ub, rhs,
                                                                                                  s->tcx_colmax.p);
  BIPB_LAUNCHED(s);
  const int64_t pk = (int64_t)n_steps * tcx::kChunks * tcx::kRHS * tcx::kKC;
  s->grow(s->tcx_upk, (size_t)n_steps * tcx::kBBytes / sizeof(float));
  __half* upk = reinterpret_cast<__half*>(s->tcx_upk.p);
  tcx::k_tcx_pack_u<<<(int)((pk + 255) / 256), 256, 0, s->stream>>>(n, nb, n_steps, ub, rhs, s->tcx_colmax.p, upk);
  BIPB_LAUNCHED(s);
  int S = 1;
  ItemPlan* plan = tcx_plan(s, n, &S);
  s->grow(s->part64, (size_t)nb * S * 2 * n);
  if (s->tc_err.cap == 0) {
    s->grow(s->tc_err, 1);
    BIPB_CUDA(cudaMemsetAsync(s->tc_err.p, 0, sizeof(int), s->stream));
  }
  auto kernel = transpose ? tcx::k_mrhs_tcx<true> : tcx::k_mrhs_tcx<false>;
  BIPB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcx::kSmemBytes));
  {
    TimedLaunch tl(s, transpose ? kTMvDFT : kTMvDF);
    kernel<<<plan->n_items, tcx::kThreads, tcx::kSmemBytes, s->stream>>>(
        n, nb, S, plan->items.p, s->geodf.p, rowexp, s->tcx_colmax.p, upk, s->part64.p, c, s->tc_err.p);
    BIPB_LAUNCHED(s);
  }
  return S;
}

}  // namespace

void matvec_df_mrhs(Surface* s, const SysLayout& L, const DFConst& c, bool transpose, const double* u, double* y,
                    double dphi, double dpsi, const int* skip, int skip_stride) {
  BIPB_REQUIRE(!transpose || s->tcx_enabled, "the multi-RHS double-float transpose runs on the tensor cores only");
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
    // 16 or more right-hand sides, or A^T: the exact tensor-core form; fewer: df64 on the CUDA cores
    const bool tensor = (nb >= kTcxMinRHS || transpose) && s->tcx_enabled;
    const int G = nb <= kGB ? 1 : nb <= 2 * kGB ? 2 : nb <= 4 * kGB ? 4 : 8;
    int S = 1;
    ItemPlan* plan = nullptr;
    if (!tensor) {
      const int slots = s->num_sms * (G == 1   ? mrhs_df_occupancy<1>()
                                      : G == 2 ? mrhs_df_occupancy<2>()
                                      : G == 4 ? mrhs_df_occupancy<4>()
                                               : mrhs_df_occupancy<8>());
      plan = mrhs_df_plan(s, n, G, slots, &S);
      s->grow(s->part64, (size_t)nb * S * 2 * n);
    }
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
    const int* rhs = nullptr;
    const double* ub = u + (int64_t)act[g0] * 2 * n;
    if (act[g0 + nb - 1] - act[g0] != nb - 1) {  // not contiguous: pass the indices
      s->grow(s->rhs_idx, (size_t)nb);
      BIPB_CUDA(cudaMemcpyAsync(s->rhs_idx.p, act.data() + g0, nb * sizeof(int), cudaMemcpyHostToDevice, s->stream));
      BIPB_CUDA(cudaStreamSynchronize(s->stream));
      rhs = s->rhs_idx.p;
      ub = u;
    }
    if (tensor) S = launch_tcx(s, n, nb, transpose, ub, rhs, c);
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
    if (tensor) {
      launch_reduce_matvec64(s, Lb, tt->second->tab.p, s->part64.p, u, y, dphi, dpsi, nullptr, 0);
      continue;
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
