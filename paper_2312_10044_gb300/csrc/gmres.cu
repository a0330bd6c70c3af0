// Device-resident restarted GMRES (Saad & Schultz; the Krylov solver of
// Sec. 2.2.2) over a batch of independent systems, and mixed-precision
// iterative refinement.
//
// Unlike the paper's GPU pipeline (Sec. 2.4), which copies x and y across
// PCIe and runs the Arnoldi process on the host every iteration, every step
// here stays on the device: mat-vec, classical Gram-Schmidt with one
// re-orthogonalisation (CGS2, the same Krylov basis as modified Gram-Schmidt
// in exact arithmetic, but as matrix-vector shaped passes; one pass for the
// FP32 Krylov solve inside the mixed modes), Givens rotations and the
// convergence test.  K systems (right-hand sides of one surface, or
// surfaces of uneven size) advance together: one Krylov vector is the
// concatenation of the K systems' vectors, every kernel covers all of them,
// and a system that has converged skips its share.  The host reads one small
// status record per system per restart cycle.  One cycle (m Arnoldi steps,
// the least-squares update and the restart vector) is recorded once as a
// CUDA graph and replayed.
//
// Restart vector: after k steps the residual of the new iterate is
// r = V_{k+1} Q^T (g_k e_{k+1}) (Q the product of the Givens rotations), so
// the next cycle starts from it without another mat-vec; the true residual
// b - A x is computed when the recurrence reports convergence.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <map>
#include <mutex>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr int kBS = 256;

struct DevState {
  int k;       // Arnoldi steps done in this cycle
  int skip;    // nonzero: the rest of the cycle does nothing for this system
  int conv;    // recurrence residual <= tol
  int stop;    // iteration cap reached
  int iters;   // Arnoldi steps in this call
  int max_iter;
  int m;
  int active;  // the system takes part in this call
  double tol;    // relative to bnorm
  double bnorm;  // norm of the right-hand side of this call
  double beta;   // norm of the current cycle's start residual
  double est;    // latest |g_k| / bnorm
  int arrive;    // blocks of this system done with the current normalisation step
  int pad_;
};
constexpr int kStateInts = (int)(sizeof(DevState) / sizeof(int));
static_assert(offsetof(DevState, skip) == sizeof(int), "skip must be the second int");

__device__ double block_sum(double v) {
  __shared__ double red[kBS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kBS / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Block table: blk[b] = {system, start, end, first block of the system},
// sysb[k] = {first block, end block, 0, 0}.  Every block covers one
// contiguous range of one system's unknowns.

// Sum of v over a warp in a fixed order (tree of shuffles down), then
// broadcast from lane 0, so every lane holds the same, reproducible value.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// sum over blocks b in [b0, b1) of part[b * stride + i], by one warp, fixed order
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part, int stride, int i, int b0, int b1) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = b0 + lane; b < b1; b += 32) s += part[(size_t)b * stride + i];
  return warp_sum(s);
}

// part[b * m1 + i] = V_i . w over block b's range, i <= j (warp i % 8 takes vector i)
__device__ __forceinline__ void block_dots(int j, int m1, int64_t len, const double* __restrict__ V,
                                           const double* w, double* __restrict__ part, int4 B) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += kBS / 32) {
    const double* v = V + (size_t)i * len;
    double acc = 0.0;
    for (int x = B.y + lane; x < B.z; x += 32) acc += v[x] * w[x];
    acc = warp_sum(acc);
    if (lane == 0) part[(size_t)blockIdx.x * m1 + i] = acc;
  }
}

// Preconditioning by the element self blocks (Sec. 2.2.4 with one element per
// leaf): with the self pair omitted, element i's 2 x 2 block of A is
// diag(1/2 (1 + eps), 1/2 (1 + 1/eps)), so M^-1 scales the phi rows by pre.x
// and the psi rows by pre.y.  It is applied on the right, A M^-1 y = r,
// d = M^-1 y: GMRES then minimises the true residual, which is what the
// stopping tests and the refinement read.  lay[k] = {geo_off, n, vec_off,
// chg_off} of system k.
__device__ __forceinline__ double precond_factor(int x, int4 Lk, double2 pre) {
  return (x - Lk.z < Lk.y) ? pre.x : pre.y;
}

__global__ void k_dots(int j, int m1, int64_t len, const double* __restrict__ V, const double* __restrict__ w,
                       double* __restrict__ part, const DevState* st, const int4* __restrict__ blk) {
  chain_wait();
  chain_release();
  const int4 B = blk[blockIdx.x];
  if (st[B.x].skip) return;
  block_dots(j, m1, len, V, w, part, B);
}

// h_i = sum over the system's blocks of part[.][i]; w -= sum_i h_i V_i; H[:, j] (+)= h;
// with want_norm, also part1[b] = sum of the updated w^2 over block b's range;
// with part_next, also the block's dot products of the updated w for the
// second Gram-Schmidt pass (block-local, so they need no extra launch).
__global__ void k_orth(int j, int m, int64_t len, const double* __restrict__ V, double* __restrict__ w,
                       const double* __restrict__ part, double* __restrict__ H, int accumulate, const DevState* st,
                       const int4* __restrict__ blk, const int4* __restrict__ sysb, double* __restrict__ part1,
                       int want_norm, double* __restrict__ part_next) {
  chain_wait();
  chain_release();
  const int4 B = blk[blockIdx.x];
  if (st[B.x].skip) return;
  const int m1 = m + 1;
  const int4 S = sysb[B.x];
  __shared__ double h[kMaxRestart + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += kBS / 32) {
    const double v = warp_sum_parts(part, m1, i, S.x, S.y);
    if (lane == 0) h[i] = v;
  }
  __syncthreads();
  if ((int)blockIdx.x == S.x) {
    double* Hs = H + (size_t)B.x * m1 * m + (size_t)j * m1;
    for (int i = threadIdx.x; i <= j; i += kBS) Hs[i] = accumulate ? Hs[i] + h[i] : h[i];
  }
  double ss = 0.0;
  for (int x = B.y + threadIdx.x; x < B.z; x += kBS) {
    double acc = w[x];
    for (int i = 0; i <= j; ++i) acc -= h[i] * V[(size_t)i * len + x];
    w[x] = acc;
    ss += acc * acc;
  }
  if (want_norm) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) part1[blockIdx.x] = ss;
  }
  if (part_next != nullptr) {
    __syncthreads();  // the block's updated w is visible to all its threads
    block_dots(j, m1, len, V, w, part_next, B);
  }
}

// part1[b] = sum of w^2 over block b's range (mode 0: systems not skipped,
// mode 1: active systems, mode 2: every system)
__global__ void k_sumsq(const double* __restrict__ w, double* __restrict__ part1, const DevState* st,
                        const int4* __restrict__ blk, int mode) {
  const int4 B = blk[blockIdx.x];
  if ((mode == 0 && st[B.x].skip) || (mode == 1 && !st[B.x].active)) return;
  double acc = 0.0;
  for (int x = B.y + threadIdx.x; x < B.z; x += kBS) acc += w[x] * w[x];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part1[blockIdx.x] = acc;
}

// Per system: apply earlier rotations to column j, make rotation j, update g,
// test.  The column (j + 2 entries, h[j + 1] = ||w||) and the earlier
// rotations are in shared memory (ch, csh, snh), staged by the caller's
// block in parallel, so the serial recurrence waits on no global load.
__device__ void givens_step(int j, int m, int sys, double* ch, const double* csh, const double* snh,
                            double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                            double* __restrict__ g, DevState* __restrict__ st) {
  DevState& S = st[sys];
  const int m1 = m + 1;
  double* h = H + (size_t)sys * m1 * m + (size_t)j * m1;
  double* g_ = g + (size_t)sys * m1;
  const double gj = g_[j], bnorm = S.bnorm, tol = S.tol;
  const int iters = S.iters + 1, max_iter = S.max_iter, Sm = S.m;
  for (int i = 0; i < j; ++i) {
    const double t = csh[i] * ch[i] + snh[i] * ch[i + 1];
    ch[i + 1] = -snh[i] * ch[i] + csh[i] * ch[i + 1];
    ch[i] = t;
  }
  const double a = ch[j], b = ch[j + 1];
  const double den = hypot(a, b);
  const double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  for (int i = 0; i < j; ++i) h[i] = ch[i];
  h[j] = den;
  h[j + 1] = 0.0;
  cs[(size_t)sys * m + j] = c;
  sn[(size_t)sys * m + j] = s;
  const double gj1 = -s * gj;
  g_[j + 1] = gj1;
  g_[j] = c * gj;
  S.k = j + 1;
  S.iters = iters;
  const double est = bnorm > 0.0 ? fabs(gj1) / bnorm : 0.0;
  S.est = est;
  const int conv = est <= tol || b == 0.0;
  const int stop = iters >= max_iter;
  if (conv) S.conv = 1;
  if (stop) S.stop = 1;
  if (conv || stop || j + 1 == Sm) S.skip = 1;
}

// out = w / ||w|| per system (and tz = M^-1 out when preconditioned); j >= 0:
// H[j+1, j] = ||w|| and the Givens step of
// column j, both by the last block of the system to finish (every block has
// then passed its skip test, so the step may set skip; the blocks' arrival
// is counted with an atomic after a fence, no block waits); j < 0: start of
// a cycle, beta = ||w|| (and bnorm = ||w|| if set_bnorm).
__global__ void k_normalize(int j, int m, const double* __restrict__ w, double* __restrict__ out,
                            const double* __restrict__ part1, double* __restrict__ H, DevState* st,
                            const int4* __restrict__ blk, const int4* __restrict__ sysb, int set_bnorm,
                            double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                            double* __restrict__ tz, const int4* __restrict__ lay, double2 pre) {
  chain_wait();
  chain_release();
  const int4 B = blk[blockIdx.x];
  if (j >= 0 ? st[B.x].skip : !st[B.x].active) return;
  const int4 S = sysb[B.x];
  __shared__ double nrm;
  if (threadIdx.x < 32) {
    const double s = warp_sum_parts(part1, 1, 0, S.x, S.y);
    if (threadIdx.x == 0) nrm = sqrt(s);
  }
  __syncthreads();
  const double v = nrm;
  const double inv = v > 0.0 ? 1.0 / v : 0.0;
  for (int x = B.y + threadIdx.x; x < B.z; x += kBS) out[x] = w[x] * inv;
  if (tz != nullptr) {  // the next mat-vec's input M^-1 out
    const int4 Lk = lay[B.x];
    for (int x = B.y + threadIdx.x; x < B.z; x += kBS) tz[x] = precond_factor(x, Lk, pre) * (w[x] * inv);
  }
  if (j < 0) {
    if (threadIdx.x == 0 && (int)blockIdx.x == S.x) {
      if (set_bnorm) st[B.x].bnorm = v;
      st[B.x].beta = v;
    }
    return;
  }
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&st[B.x].arrive, 1) == S.y - S.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double ch[kMaxRestart + 1], csh[kMaxRestart], snh[kMaxRestart];
  const double* Hc = H + (size_t)B.x * (m + 1) * m + (size_t)j * (m + 1);
  for (int i = threadIdx.x; i <= j; i += kBS) ch[i] = Hc[i];
  for (int i = threadIdx.x; i < j; i += kBS) csh[i] = cs[(size_t)B.x * m + i], snh[i] = sn[(size_t)B.x * m + i];
  if (threadIdx.x == 0) ch[j + 1] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  st[B.x].arrive = 0;
  givens_step(j, m, B.x, ch, csh, snh, H, cs, sn, g, st);
}

// Per system: least squares R y = g (k x k) and the restart coefficients
// z = Q^T (g_k e_k) / |g_k|.
__global__ void k_lsq(int m, int K, const double* __restrict__ H, const double* __restrict__ cs,
                      const double* __restrict__ sn, const double* __restrict__ g, double* __restrict__ y,
                      double* __restrict__ z, DevState* st) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= K) return;
  DevState& S = st[sys];
  const int k = S.k;
  if (!S.active || k == 0) return;
  const int m1 = m + 1;
  const double* Hs = H + (size_t)sys * m1 * m;
  const double* c_ = cs + (size_t)sys * m;
  const double* s_ = sn + (size_t)sys * m;
  const double* g_ = g + (size_t)sys * m1;
  double* y_ = y + (size_t)sys * m;
  double* z_ = z + (size_t)sys * m1;
  for (int i = k - 1; i >= 0; --i) {
    double s = g_[i];
    for (int l = i + 1; l < k; ++l) s -= Hs[(size_t)l * m1 + i] * y_[l];
    y_[i] = s / Hs[(size_t)i * m1 + i];
  }
  const double gk = g_[k];
  const double beta = fabs(gk);
  for (int i = 0; i <= k; ++i) z_[i] = 0.0;
  z_[k] = beta > 0.0 ? gk / beta : 0.0;
  for (int i = k - 1; i >= 0; --i) {
    double a = z_[i], b = z_[i + 1];
    z_[i] = c_[i] * a - s_[i] * b;
    z_[i + 1] = s_[i] * a + c_[i] * b;
  }
  S.beta = beta;
}

// x += M^-1 sum_{i<k} y_i V_i ; V_0 <- sum_{i<=k} z_i V_i (per system); when
// preconditioned (tz != nullptr) also tz = M^-1 V_0, the next cycle's first input
__global__ void k_update(int m, int64_t len, double* __restrict__ V, double* __restrict__ x,
                         const double* __restrict__ y, const double* __restrict__ z, const DevState* st,
                         const int4* __restrict__ blk, double* __restrict__ tz, const int4* __restrict__ lay,
                         double2 pre) {
  const int4 B = blk[blockIdx.x];
  const DevState& S = st[B.x];
  const int k = S.k;
  if (!S.active || k == 0) return;
  const double* y_ = y + (size_t)B.x * m;
  const double* z_ = z + (size_t)B.x * (m + 1);
  for (int e = B.y + threadIdx.x; e < B.z; e += kBS) {
    double dx = 0.0, v0 = 0.0;
    for (int i = 0; i <= k; ++i) {
      double v = V[(size_t)i * len + e];
      if (i < k) dx += y_[i] * v;
      v0 += z_[i] * v;
    }
    if (tz != nullptr) {
      const double f = precond_factor(e, lay[B.x], pre);
      x[e] += f * dx;
      tz[e] = f * v0;
    } else {
      x[e] += dx;
    }
    V[e] = v0;
  }
}

__global__ void k_next_cycle(int m, int K, double* __restrict__ g, DevState* st) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= K) return;
  DevState& S = st[sys];
  if (!S.active) return;
  double* g_ = g + (size_t)sys * (m + 1);
  g_[0] = S.beta;
  for (int i = 1; i <= m; ++i) g_[i] = 0.0;
  S.k = 0;
  S.est = S.bnorm > 0.0 ? S.beta / S.bnorm : 0.0;
  if (S.beta == 0.0 || S.est <= S.tol) S.conv = 1;
  S.skip = (S.conv || S.stop) ? 1 : 0;
}

__global__ void k_sub(int64_t len, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * kBS + threadIdx.x;
  if (i < len) out[i] = a[i] - b[i];
}
__global__ void k_add(int64_t len, const double* __restrict__ a, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * kBS + threadIdx.x;
  if (i < len) out[i] += a[i];
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, (n + kBS - 1) / kBS); }

struct GraphTag {
  uint64_t gen;
  double eps_in, eps_out, kappa;
  bool timed;
  bool operator==(const GraphTag& o) const {
    return gen == o.gen && eps_in == o.eps_in && eps_out == o.eps_out && kappa == o.kappa && timed == o.timed;
  }
};
struct Recorded {
  cudaGraphExec_t exec;
  GraphTag tag;
  std::vector<EventPair> events;  // timing events recorded inside the graph
  long long kernels;              // kernel nodes in the graph
};

}  // namespace

struct GmresWork {
  uint64_t lay_key = 0;
  int m = 0, K = 0, nblk = 0;
  int precond = 0;  // bipb_precond of the current call
  int64_t len = 0;
  DevBuf<double> V, w, H, cs, sn, g, y, z, part, part2, part1, r, d, t, tz;
  DevBuf<int4> blk, sysb;
  DevBuf<int> mask;  // per system: 1 = leave out of the FP64 residual
  std::vector<int4> sysb_host;
  DevBuf<DevState> st_buf;
  DevState* st = nullptr;  // st_buf.p
  // host copies (pageable: every transfer of them is followed by a synchronisation)
  std::vector<DevState> st_host;
  std::vector<double> part1_host;
  std::vector<int> mask_host;
  std::map<int, Recorded> graphs;  // recorded cycles keyed by (precision, transpose, precond)
  const std::vector<EventPair>* replayed = nullptr;
  int device = 0;
  ~GmresWork();
};

namespace {

// Executable restart-cycle graphs of destroyed handles, kept for reuse: a new
// handle records its own cycle and, when a kept executable of the same kind
// accepts that graph (cudaGraphExecUpdate checks that the topology matches),
// updates it in place instead of instantiating a new one.  At most kPoolMax
// are kept; they are released with the process (the pool is never destroyed,
// so no CUDA call runs during static destruction).
struct PooledExec {
  int device, key;
  cudaGraphExec_t exec;
};
constexpr size_t kPoolMax = 16;
std::mutex& pool_mutex() {
  static auto* m = new std::mutex;
  return *m;
}
std::vector<PooledExec>& exec_pool() {
  static auto* v = new std::vector<PooledExec>;
  return *v;
}

void pool_put(int device, int key, cudaGraphExec_t exec) {
  std::lock_guard<std::mutex> lock(pool_mutex());
  if (exec_pool().size() < kPoolMax) {
    exec_pool().push_back(PooledExec{device, key, exec});
  } else {
    cudaGraphExecDestroy(exec);
  }
}

// An executable updated to run graph g, or nullptr.
cudaGraphExec_t pool_take(int device, int key, cudaGraph_t g) {
  std::lock_guard<std::mutex> lock(pool_mutex());
  auto& v = exec_pool();
  int tries = 0;
  for (size_t i = 0; i < v.size() && tries < 4; ++i) {
    if (v[i].device != device || v[i].key != key) continue;
    ++tries;
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(v[i].exec, g, &info) == cudaSuccess) {
      cudaGraphExec_t e = v[i].exec;
      v.erase(v.begin() + (std::ptrdiff_t)i);
      return e;
    }
    (void)cudaGetLastError();  // a topology mismatch is not an error here
  }
  return nullptr;
}

}  // namespace

GmresWork::~GmresWork() {
  for (auto& kv : graphs) {
    if (kv.second.events.empty()) {
      pool_put(device, kv.first, kv.second.exec);  // untimed cycles only: no event nodes to carry over
    } else {
      cudaGraphExecDestroy(kv.second.exec);
      for (auto& e : kv.second.events) cudaEventDestroy(e.a), cudaEventDestroy(e.b);
    }
  }
}

void gmres_free(Surface* s) {
  delete s->gw;
  s->gw = nullptr;
}

namespace {

GmresWork* workspace(Surface* s, const SysLayout& L, int m) {
  GmresWork* w = s->gw;
  if (w && w->lay_key == L.key && w->m == m && w->K == L.K) return w;
  if (w) gmres_free(s);
  w = new GmresWork();
  w->device = s->device;
  s->gw = w;
  w->lay_key = L.key;
  w->m = m;
  w->K = L.K;
  w->len = L.len;
  // blocks: each covers one contiguous range (about 256 unknowns, at most
  // 1024 blocks per system) of one system
  std::vector<int4> blk;
  std::vector<int4> sysb(L.K);
  for (int k = 0; k < L.K; ++k) {
    const int64_t lk = 2 * (int64_t)L.n[k];
    const int nb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (lk + 255) / 256));
    const int64_t chunk = (lk + nb - 1) / nb;
    sysb[k] = make_int4((int)blk.size(), (int)blk.size() + nb, 0, 0);
    for (int b = 0; b < nb; ++b) {
      const int64_t a = L.vec_off[k] + b * chunk, e = std::min<int64_t>(L.vec_off[k] + lk, a + chunk);
      blk.push_back(make_int4(k, (int)a, (int)e, sysb[k].x));
    }
  }
  w->nblk = (int)blk.size();
  w->sysb_host = sysb;
  const int64_t len = L.len;
  w->V.ensure((size_t)(m + 1) * len, s->stream);
  w->w.ensure(len, s->stream);
  w->r.ensure(len, s->stream);
  w->d.ensure(len, s->stream);
  w->tz.ensure(len, s->stream);
  w->t.ensure(len, s->stream);
  w->H.ensure((size_t)L.K * (m + 1) * m, s->stream);
  w->cs.ensure((size_t)L.K * m, s->stream);
  w->sn.ensure((size_t)L.K * m, s->stream);
  w->g.ensure((size_t)L.K * (m + 1), s->stream);
  w->y.ensure((size_t)L.K * m, s->stream);
  w->z.ensure((size_t)L.K * (m + 1), s->stream);
  w->part.ensure((size_t)w->nblk * (m + 1), s->stream);
  w->part2.ensure((size_t)w->nblk * (m + 1), s->stream);
  w->part1.ensure(w->nblk, s->stream);
  w->blk.ensure(blk.size(), s->stream);
  w->sysb.ensure(L.K, s->stream);
  w->mask.ensure(L.K, s->stream);
  w->st_buf.ensure(L.K, s->stream);
  w->st = w->st_buf.p;
  w->st_host.resize(L.K);
  w->part1_host.resize(w->nblk);
  w->mask_host.resize(L.K);
  BIPB_CUDA(cudaMemcpyAsync(w->blk.p, blk.data(), blk.size() * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
  BIPB_CUDA(cudaMemcpyAsync(w->sysb.p, sysb.data(), sysb.size() * sizeof(int4), cudaMemcpyHostToDevice, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  ++s->alloc_gen;
  return w;
}

// One restart cycle: kernels only (no host synchronisation, no allocation).
// M^-1 of the self-block preconditioner: 1 / (1/2 (1 + eps)), 1 / (1/2 (1 + 1/eps))
double2 precond_factors(const bipb_medium& m) {
  const double eps = m.eps_out / m.eps_in;
  return make_double2(2.0 / (1.0 + eps), 2.0 / (1.0 + 1.0 / eps));
}

void issue_cycle(Surface* s, const SysLayout& L, GmresWork* w, const bipb_medium& med, int precision,
                 bool transpose) {
  const int4* lay = w->precond ? s->lay_dev(L) : nullptr;
  double* tz = w->precond ? w->tz.p : nullptr;
  const double2 pre = precond_factors(med);
  const int m = w->m, m1 = m + 1, K = w->K, nb = w->nblk;
  const int64_t len = w->len;
  const int kg = (K + 127) / 128;
  const bool cgs2 = precision == BIPB_FP64 || precision == BIPB_DF64;
  for (int j = 0; j < m; ++j) {
    double* vj = w->V.p + (size_t)j * len;
    matvec(s, L, med, precision, transpose, tz ? tz : vj, w->w.p, &w->st->skip, kStateInts);
    // CGS2 for FP64 and df64 Krylov mat-vecs: the first pass also takes the
    // dot products of the second, the second also forms the block norms.
    // The FP32 / split-FP16 tensor-core Krylov solve of the mixed modes stops at a
    // relative 1e-6 (its true residual is measured in higher precision by
    // the refinement), and its FP64 basis of at most m vectors loses
    // orthogonality in one classical pass only at about eps_64 cond(A)^2:
    // one pass, which also forms the block norms.
    launch_chained(k_dots, nb, kBS, 0, s->stream, j, m1, len, w->V.p, w->w.p, w->part.p, w->st, w->blk.p);
    BIPB_LAUNCHED(s);
    if (cgs2) {
      launch_chained(k_orth, nb, kBS, 0, s->stream, j, m, len, w->V.p, w->w.p, w->part.p, w->H.p, 0, w->st, w->blk.p,
                     w->sysb.p, w->part1.p, 0, w->part2.p);
      BIPB_LAUNCHED(s);
      launch_chained(k_orth, nb, kBS, 0, s->stream, j, m, len, w->V.p, w->w.p, w->part2.p, w->H.p, 1, w->st,
                     w->blk.p, w->sysb.p, w->part1.p, 1, nullptr);
    } else {
      launch_chained(k_orth, nb, kBS, 0, s->stream, j, m, len, w->V.p, w->w.p, w->part.p, w->H.p, 0, w->st, w->blk.p,
                     w->sysb.p, w->part1.p, 1, nullptr);
    }
    BIPB_LAUNCHED(s);
    launch_chained(k_normalize, nb, kBS, 0, s->stream, j, m, w->w.p, vj + len, w->part1.p, w->H.p, w->st, w->blk.p,
                   w->sysb.p, 0, w->cs.p, w->sn.p, w->g.p, tz, lay, pre);
    BIPB_LAUNCHED(s);
  }
  k_lsq<<<kg, 128, 0, s->stream>>>(m, K, w->H.p, w->cs.p, w->sn.p, w->g.p, w->y.p, w->z.p, w->st);
  BIPB_LAUNCHED(s);
  k_update<<<nb, kBS, 0, s->stream>>>(m, len, w->V.p, w->d.p, w->y.p, w->z.p, w->st, w->blk.p, tz, lay, pre);
  BIPB_LAUNCHED(s);
  k_next_cycle<<<kg, 128, 0, s->stream>>>(m, K, w->g.p, w->st);
  BIPB_LAUNCHED(s);
}

void run_cycle(Surface* s, const SysLayout& L, GmresWork* w, const bipb_medium& med, int precision,
               bool transpose) {
  // A recorded cycle bakes in the medium and every buffer address, so it is
  // tagged with both and re-recorded when either changes.
  const int key = (precision * 2 + (transpose ? 1 : 0)) * 2 + (w->precond ? 1 : 0);
  const GraphTag tag{s->alloc_gen, med.eps_in, med.eps_out, med.kappa, s->timer.on};
  auto it = w->graphs.find(key);
  if (it != w->graphs.end() && it->second.tag == tag) {
    BIPB_CUDA(cudaGraphLaunch(it->second.exec, s->stream));
    s->launches += it->second.kernels;
    w->replayed = &it->second.events;
    return;
  }
  // a plain launch first: it runs this cycle and creates every scratch buffer
  issue_cycle(s, L, w, med, precision, transpose);
  const GraphTag after{s->alloc_gen, med.eps_in, med.eps_out, med.kappa, s->timer.on};
  // record a copy of the cycle for the next calls (recording does not run it)
  cudaGraph_t graph = nullptr;
  std::vector<EventPair> evs;
  BIPB_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  s->timer.capture = &evs;
  s->recording = true;
  s->recorded_launches = 0;
  try {
    issue_cycle(s, L, w, med, precision, transpose);
  } catch (...) {
    s->recording = false;
    s->timer.capture = nullptr;
    cudaStreamEndCapture(s->stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  s->timer.capture = nullptr;
  s->recording = false;
  const long long kernels = s->recorded_launches;
  BIPB_CUDA(cudaStreamEndCapture(s->stream, &graph));
  if (!(s->alloc_gen == after.gen)) {  // a buffer moved while recording: do not keep it
    cudaGraphDestroy(graph);
    for (auto& e : evs) s->timer.pool.push_back(e.a), s->timer.pool.push_back(e.b);
    return;
  }
  cudaGraphExec_t exec = evs.empty() ? pool_take(s->device, key, graph) : nullptr;
  cudaError_t e = exec ? cudaSuccess : cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  BIPB_CUDA(e);
  if (it != w->graphs.end()) {
    cudaGraphExecDestroy(it->second.exec);
    for (auto& ev : it->second.events) s->timer.pool.push_back(ev.a), s->timer.pool.push_back(ev.b);
  }
  w->graphs[key] = Recorded{exec, after, std::move(evs), kernels};
}

void read_states(Surface* s, GmresWork* w) {
  BIPB_CUDA(cudaMemcpyAsync(w->st_host.data(), w->st, w->K * sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  if (s->timer.on) {
    s->timer.collect();
    if (w->replayed)
      for (auto& e : *w->replayed) s->timer.add(e);
  }
  w->replayed = nullptr;
}

// Per-system 2-norms of a batched vector (all systems, fixed summation order).
std::vector<double> norms(Surface* s, GmresWork* w, const double* v) {
  k_sumsq<<<w->nblk, kBS, 0, s->stream>>>(v, w->part1.p, w->st, w->blk.p, 2);
  BIPB_LAUNCHED(s);
  BIPB_CUDA(cudaMemcpyAsync(w->part1_host.data(), w->part1.p, w->nblk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<double> out(w->K);
  for (int k = 0; k < w->K; ++k) {
    double acc = 0.0;
    for (int b = w->sysb_host[k].x; b < w->sysb_host[k].y; ++b) acc += w->part1_host[b];
    out[k] = std::sqrt(acc);
  }
  return out;
}

// GMRES on op(A) d = r0 for the active systems (d starts at zero; others are
// left alone).  Per system: stop at recurrence estimate <= tol[k] (relative
// to ||r0_k||) or after cap[k] iterations.  Returns iterations per system.
std::vector<int> gmres_core(Surface* s, const SysLayout& L, GmresWork* w, const bipb_medium& med, int precision,
                            bool transpose, const double* r0, const std::vector<char>& active,
                            const std::vector<double>& tol, const std::vector<int>& cap, std::vector<int>* conv) {
  const int K = w->K;
  BIPB_CUDA(cudaMemsetAsync(w->d.p, 0, (size_t)w->len * sizeof(double), s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));  // st_host is about to be rewritten
  for (int k = 0; k < K; ++k) {
    DevState& S = w->st_host[k];
    S = DevState{};
    S.active = active[k] ? 1 : 0;
    S.skip = S.active ? 0 : 1;
    S.conv = S.active ? 0 : 1;
    S.stop = (S.active && cap[k] <= 0) ? 1 : 0;
    S.max_iter = cap[k];
    S.m = w->m;
    S.tol = tol[k];
    S.est = 1.0;
  }
  BIPB_CUDA(cudaMemcpyAsync(w->st, w->st_host.data(), K * sizeof(DevState), cudaMemcpyHostToDevice, s->stream));
  const int kg = (K + 127) / 128;
  k_sumsq<<<w->nblk, kBS, 0, s->stream>>>(r0, w->part1.p, w->st, w->blk.p, 1);
  BIPB_LAUNCHED(s);
  k_normalize<<<w->nblk, kBS, 0, s->stream>>>(-1, w->m, r0, w->V.p, w->part1.p, w->H.p, w->st, w->blk.p, w->sysb.p,
                                              1, w->cs.p, w->sn.p, w->g.p, w->precond ? w->tz.p : nullptr,
                                              w->precond ? s->lay_dev(L) : nullptr, precond_factors(med));
  BIPB_LAUNCHED(s);
  k_next_cycle<<<kg, 128, 0, s->stream>>>(w->m, K, w->g.p, w->st);
  BIPB_LAUNCHED(s);
  read_states(s, w);
  auto running = [&] {
    for (int k = 0; k < K; ++k)
      if (w->st_host[k].active && !w->st_host[k].conv && !w->st_host[k].stop) return true;
    return false;
  };
  while (running()) {
    run_cycle(s, L, w, med, precision, transpose);
    read_states(s, w);
  }
  std::vector<int> it(K);
  conv->assign(K, 0);
  for (int k = 0; k < K; ++k) {
    it[k] = w->st_host[k].iters;
    (*conv)[k] = w->st_host[k].conv;
  }
  return it;
}

}  // namespace

std::vector<SolveResult> gmres_solve(Surface* s, const SysLayout& L, const bipb_medium& med,
                                     const bipb_solve_params& p, bool transpose, const double* rhs, double* x,
                                     bool warm) {
  const int K = L.K;
  std::vector<SolveResult> res(K);
  const int m = p.restart > 0 ? p.restart : 10;
  const int max_iter = p.max_iter > 0 ? p.max_iter : 1000;
  GmresWork* w = workspace(s, L, m);
  w->precond = p.precond;
  const int64_t len = L.len;
  const int nb = grid_for(len);
  const std::vector<double> bnorm = norms(s, w, rhs);
  const bool mixed = p.precision == BIPB_MIXED || p.precision == BIPB_MIXED_DF64 || p.precision == BIPB_MIXED_TENSOR ||
                     p.precision == BIPB_MIXED_TREE;
  // arithmetic of the Krylov mat-vecs and of the residual r = b - A x
  int inner = !mixed ? p.precision : BIPB_FP32;
  if (p.precision == BIPB_MIXED_TENSOR) inner = BIPB_TENSOR;
  if (p.precision == BIPB_MIXED_TREE) inner = BIPB_TREE32;
  const int resid = (p.precision == BIPB_MIXED || p.precision == BIPB_FP64) ? BIPB_FP64 : BIPB_DF64;
  // r = rhs - A x (or rhs when starting from zero)
  if (warm) {
    matvec(s, L, med, resid, transpose, x, w->t.p, nullptr, 0);
    for (auto& r : res) r.matvecs64++;
    k_sub<<<nb, kBS, 0, s->stream>>>(len, rhs, w->t.p, w->r.p);
    BIPB_LAUNCHED(s);
  } else {
    BIPB_CUDA(cudaMemsetAsync(x, 0, (size_t)len * sizeof(double), s->stream));
    BIPB_CUDA(cudaMemcpyAsync(w->r.p, rhs, (size_t)len * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  }
  std::vector<double> rel(K, 1.0);
  if (warm) {
    std::vector<double> rn = norms(s, w, w->r.p);
    for (int k = 0; k < K; ++k) rel[k] = bnorm[k] > 0 ? rn[k] / bnorm[k] : 0.0;
  }
  for (int k = 0; k < K; ++k)
    if (bnorm[k] == 0.0) rel[k] = 0.0;
  // inner solves stop near the inner operator's own accuracy (about 1e-7 for
  // FP32 pairs and for the split-FP16 tensor-core tiles): iterating further
  // does not reduce the true residual
  const double inner_floor = p.inner_tol > 0 ? p.inner_tol : 1e-6;
  const int inner_cap = p.inner_max_iter > 0 ? p.inner_max_iter : 200;
  std::vector<char> active(K), done(K, 0);
  std::vector<int> iters(K, 0);
  for (;;) {
    bool any = false;
    std::vector<double> tol_rel(K, 1.0);
    std::vector<int> cap(K, 0);
    for (int k = 0; k < K; ++k) {
      active[k] = !done[k] && rel[k] > p.tol && iters[k] < max_iter;
      if (!active[k]) continue;
      any = true;
      cap[k] = max_iter - iters[k];
      if (mixed) {
        tol_rel[k] = std::max(inner_floor, 0.3 * p.tol / rel[k]);
        cap[k] = std::min(cap[k], inner_cap);
      } else {
        tol_rel[k] = p.tol / rel[k];
      }
    }
    if (!any) break;
    std::vector<int> conv;
    std::vector<int> used = gmres_core(s, L, w, med, inner, transpose, w->r.p, active, tol_rel, cap, &conv);
    // x += d (d is zero outside the active systems); r = rhs - A x in FP64 for the active systems
    k_add<<<nb, kBS, 0, s->stream>>>(len, w->d.p, x);
    BIPB_LAUNCHED(s);
    for (int k = 0; k < K; ++k) w->mask_host[k] = active[k] ? 0 : 1;
    BIPB_CUDA(cudaMemcpyAsync(w->mask.p, w->mask_host.data(), K * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    matvec(s, L, med, resid, transpose, x, w->t.p, w->mask.p, 1);
    k_sub<<<nb, kBS, 0, s->stream>>>(len, rhs, w->t.p, w->r.p);
    BIPB_LAUNCHED(s);
    std::vector<double> rn = norms(s, w, w->r.p);
    for (int k = 0; k < K; ++k) {
      if (!active[k]) continue;
      iters[k] += used[k];
      res[k].matvecs64++;
      if (mixed) {
        res[k].matvecs32 += used[k];
        res[k].refine_steps++;
      } else {
        res[k].matvecs64 += used[k];
      }
      const double new_rel = bnorm[k] > 0 ? rn[k] / bnorm[k] : 0.0;
      if (!mixed && !conv[k]) done[k] = 1;                                           // iteration cap
      if (mixed && res[k].refine_steps >= 3 && new_rel > 0.1 * rel[k]) done[k] = 1;  // refinement stalled
      rel[k] = new_rel;
    }
  }
  for (int k = 0; k < K; ++k) {
    res[k].iters = iters[k];
    res[k].rel_residual = rel[k];
    res[k].converged = rel[k] <= p.tol ? 1 : 0;
  }
  return res;
}

}  // namespace bipb
