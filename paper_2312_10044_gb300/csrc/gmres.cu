// Device-resident restarted GMRES (Saad & Schultz; the Krylov solver of
// Sec. 2.2.2) and mixed-precision iterative refinement.
//
// Unlike the paper's GPU pipeline (Sec. 2.4), which copies x and y across
// PCIe and runs the Arnoldi process on the host every iteration, every step
// here stays on the device: mat-vec, classical Gram-Schmidt with one
// re-orthogonalisation (CGS2, the same Krylov basis as modified Gram-Schmidt
// in exact arithmetic, but as matrix-vector shaped passes), Givens rotations
// and the convergence test.  The host reads one small status record per
// restart cycle.  One cycle (m Arnoldi steps, the least-squares update and
// the restart vector) is recorded once as a CUDA graph and replayed.
//
// Restart vector: after k steps the residual of the new iterate is
// r = V_{k+1} Q^T (g_k e_{k+1}) (Q the product of the Givens rotations), so
// the next cycle starts from it without another mat-vec; the true residual
// b - A x is computed once when the recurrence reports convergence.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr int kBS = 256;

struct DevState {
  int k;        // Arnoldi steps done in this cycle
  int skip;     // nonzero: the rest of the cycle does nothing
  int conv;     // recurrence residual <= tol
  int stop;     // iteration cap reached
  int iters;    // total Arnoldi steps
  int max_iter;
  int m;
  int pad;
  double tol;    // relative to bnorm
  double bnorm;  // ||rhs||
  double beta;   // norm of the current cycle's start residual
  double est;    // latest |g_k| / bnorm
};

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

// part[blockIdx.x * (m+1) + i] = sum over this block's range of V_i . w, i <= j
__global__ void k_dots(int len, int j, int m1, const double* __restrict__ V, const double* __restrict__ w,
                       double* __restrict__ part, const DevState* st) {
  if (st->skip) return;
  for (int i = 0; i <= j; ++i) {
    const double* v = V + (size_t)i * len;
    double acc = 0.0;
    for (int x = blockIdx.x * kBS + threadIdx.x; x < len; x += gridDim.x * kBS) acc += v[x] * w[x];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x * m1 + i] = acc;
  }
}

// h_i = sum_b part[b][i]; w -= sum_i h_i V_i; H[:, j] (+)= h
__global__ void k_orth(int len, int j, int m1, int nblk, const double* __restrict__ V, double* __restrict__ w,
                       const double* __restrict__ part, double* __restrict__ H, int accumulate,
                       const DevState* st) {
  if (st->skip) return;
  __shared__ double h[kMaxRestart + 1];
  for (int i = threadIdx.x; i <= j; i += kBS) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b * m1 + i];
    h[i] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= j; i += kBS) H[(size_t)j * m1 + i] = accumulate ? H[(size_t)j * m1 + i] + h[i] : h[i];
  for (int x = blockIdx.x * kBS + threadIdx.x; x < len; x += gridDim.x * kBS) {
    double acc = w[x];
    for (int i = 0; i <= j; ++i) acc -= h[i] * V[(size_t)i * len + x];
    w[x] = acc;
  }
}

__global__ void k_sumsq(int len, const double* __restrict__ w, double* __restrict__ part, const DevState* st,
                        int ignore_skip) {
  if (!ignore_skip && st->skip) return;
  double acc = 0.0;
  for (int x = blockIdx.x * kBS + threadIdx.x; x < len; x += gridDim.x * kBS) acc += w[x] * w[x];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// out = w / ||w|| with ||w||^2 = sum_b part[b]; H[j+1, j] = ||w|| (j >= 0), or
// start a cycle (j < 0): beta = ||w||, bnorm set if requested.
__global__ void k_normalize(int len, int j, int m1, int nblk, const double* __restrict__ w,
                            double* __restrict__ out, const double* __restrict__ part, double* __restrict__ H,
                            DevState* st, int set_bnorm) {
  if (j >= 0 && st->skip) return;
  __shared__ double nrm;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b];
    nrm = sqrt(s);
  }
  __syncthreads();
  const double v = nrm;
  const double inv = v > 0.0 ? 1.0 / v : 0.0;
  for (int x = blockIdx.x * kBS + threadIdx.x; x < len; x += gridDim.x * kBS) out[x] = w[x] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (j >= 0) {
      H[(size_t)j * m1 + j + 1] = v;
    } else {
      if (set_bnorm) st->bnorm = v;
      st->beta = v;
    }
  }
}

// Apply earlier rotations to column j, make rotation j, update g, test.
__global__ void k_givens(int j, int m1, double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, DevState* st) {
  if (st->skip) return;
  double* h = H + (size_t)j * m1;
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
    h[i] = t;
  }
  double a = h[j], b = h[j + 1];
  double den = hypot(a, b);
  double c = den > 0.0 ? a / den : 1.0, s = den > 0.0 ? b / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  h[j] = den;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  st->k = j + 1;
  st->iters += 1;
  st->est = st->bnorm > 0.0 ? fabs(g[j + 1]) / st->bnorm : 0.0;
  if (st->est <= st->tol || b == 0.0) st->conv = 1;
  if (st->iters >= st->max_iter) st->stop = 1;
  if (st->conv || st->stop || j + 1 == st->m) st->skip = 1;
}

// Least squares R y = g (k x k) and the restart coefficients z = Q^T (g_k e_k) / |g_k|.
__global__ void k_lsq(int m1, const double* __restrict__ H, const double* __restrict__ cs,
                      const double* __restrict__ sn, const double* __restrict__ g, double* __restrict__ y,
                      double* __restrict__ z, DevState* st) {
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * m1 + i] * y[l];
    y[i] = s / H[(size_t)i * m1 + i];
  }
  double gk = g[k];
  double beta = fabs(gk);
  for (int i = 0; i <= k; ++i) z[i] = 0.0;
  z[k] = beta > 0.0 ? gk / beta : 0.0;
  for (int i = k - 1; i >= 0; --i) {
    double a = z[i], b = z[i + 1];
    z[i] = cs[i] * a - sn[i] * b;
    z[i + 1] = sn[i] * a + cs[i] * b;
  }
  st->beta = beta;
}

// x += sum_{i<k} y_i V_i ; V_0 <- sum_{i<=k} z_i V_i ; next cycle's g, k, skip.
__global__ void k_update(int len, int m1, double* __restrict__ V, double* __restrict__ x,
                         const double* __restrict__ y, const double* __restrict__ z, double* __restrict__ g,
                         DevState* st) {
  const int k = st->k;
  for (int e = blockIdx.x * kBS + threadIdx.x; e < len; e += gridDim.x * kBS) {
    double dx = 0.0, v0 = 0.0;
    for (int i = 0; i <= k; ++i) {
      double v = V[(size_t)i * len + e];
      if (i < k) dx += y[i] * v;
      v0 += z[i] * v;
    }
    x[e] += dx;
    V[e] = v0;
  }
}

__global__ void k_next_cycle(int m1, double* __restrict__ g, DevState* st) {
  g[0] = st->beta;
  for (int i = 1; i < m1; ++i) g[i] = 0.0;
  st->k = 0;
  st->est = st->bnorm > 0.0 ? st->beta / st->bnorm : 0.0;
  if (st->beta == 0.0 || st->est <= st->tol) st->conv = 1;
  st->skip = (st->conv || st->stop) ? 1 : 0;
}

// r = rhs - y (2n), elementwise
__global__ void k_sub(int len, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  int i = blockIdx.x * kBS + threadIdx.x;
  if (i < len) out[i] = a[i] - b[i];
}
__global__ void k_axpy(int len, double alpha, const double* __restrict__ a, double* __restrict__ out) {
  int i = blockIdx.x * kBS + threadIdx.x;
  if (i < len) out[i] += alpha * a[i];
}
__global__ void k_init_state(DevState* st, int m, int max_iter, double tol) {
  st->k = 0;
  st->skip = 0;
  st->conv = 0;
  st->stop = max_iter <= 0 ? 1 : 0;
  st->iters = 0;
  st->max_iter = max_iter;
  st->m = m;
  st->tol = tol;
  st->est = 1.0;
}

}  // namespace

struct GraphTag {
  uint64_t gen;
  double eps_in, eps_out, kappa;
  bool operator==(const GraphTag& o) const {
    return gen == o.gen && eps_in == o.eps_in && eps_out == o.eps_out && kappa == o.kappa;
  }
};
struct Recorded {
  cudaGraphExec_t exec;
  GraphTag tag;
  std::vector<EventPair> events;  // timing events recorded inside the graph
  long long kernels;              // kernel nodes in the graph
};

struct GmresWork {
  int64_t n = 0;
  int m = 0;
  int nblk = 0;
  DevBuf<double> V, w, H, cs, sn, g, y, z, part, r, d, t;
  DevState* st = nullptr;     // device
  DevState* st_host = nullptr;  // pinned
  // recorded cycles keyed by (precision, transpose)
  std::map<int, Recorded> graphs;
  const std::vector<EventPair>* replayed = nullptr;  // events of the graph launched last
  ~GmresWork() {
    for (auto& kv : graphs) {
      cudaGraphExecDestroy(kv.second.exec);
      for (auto& e : kv.second.events) cudaEventDestroy(e.a), cudaEventDestroy(e.b);
    }
    if (st) cudaFree(st);
    if (st_host) cudaFreeHost(st_host);
  }
};

void gmres_free(Surface* s) {
  delete s->gw;
  s->gw = nullptr;
}

namespace {

GmresWork* workspace(Surface* s, int m) {
  GmresWork* w = s->gw;
  if (w && w->n == s->n && w->m == m) return w;
  if (w) gmres_free(s);
  w = new GmresWork();
  s->gw = w;
  const int64_t len = 2 * s->n;
  w->n = s->n;
  w->m = m;
  w->nblk = (int)std::min<int64_t>(2 * s->num_sms, (len + 4 * kBS - 1) / (4 * kBS));
  w->nblk = std::max(w->nblk, 1);
  w->V.ensure((size_t)(m + 1) * len);
  w->w.ensure(len);
  w->r.ensure(len);
  w->d.ensure(len);
  w->t.ensure(len);
  w->H.ensure((size_t)(m + 1) * m);
  w->cs.ensure(m);
  w->sn.ensure(m);
  w->g.ensure(m + 1);
  w->y.ensure(m);
  w->z.ensure(m + 1);
  w->part.ensure((size_t)w->nblk * (m + 1));
  BIPB_CUDA(cudaMalloc(reinterpret_cast<void**>(&w->st), sizeof(DevState)));
  BIPB_CUDA(cudaMallocHost(reinterpret_cast<void**>(&w->st_host), sizeof(DevState)));
  return w;
}

int blocks(int64_t n) { return (int)((n + kBS - 1) / kBS); }

// Norm of vec into st->beta (and bnorm if set_bnorm), out = vec / ||vec||.
void start_cycle(Surface* s, GmresWork* w, const double* vec, bool set_bnorm) {
  const int len = (int)(2 * s->n);
  k_sumsq<<<w->nblk, kBS, 0, s->stream>>>(len, vec, w->part.p, w->st, 1);
  BIPB_LAUNCHED(s);
  k_normalize<<<w->nblk, kBS, 0, s->stream>>>(len, -1, w->m + 1, w->nblk, vec, w->V.p, w->part.p, w->H.p,
                                               w->st, set_bnorm ? 1 : 0);
  BIPB_LAUNCHED(s);
  k_next_cycle<<<1, 1, 0, s->stream>>>(w->m + 1, w->g.p, w->st);
  BIPB_LAUNCHED(s);
}

// One restart cycle: kernels only (no host synchronisation, no allocation).
void issue_cycle(Surface* s, GmresWork* w, const bipb_medium& med, int precision, bool transpose) {
  const int len = (int)(2 * s->n);
  const int m = w->m, m1 = m + 1;
  for (int j = 0; j < m; ++j) {
    double* vj = w->V.p + (size_t)j * len;
    matvec(s, med, precision, transpose, vj, w->w.p, &w->st->skip);
    for (int pass = 0; pass < 2; ++pass) {
      k_dots<<<w->nblk, kBS, 0, s->stream>>>(len, j, m1, w->V.p, w->w.p, w->part.p, w->st);
      BIPB_LAUNCHED(s);
      k_orth<<<w->nblk, kBS, 0, s->stream>>>(len, j, m1, w->nblk, w->V.p, w->w.p, w->part.p, w->H.p, pass,
                                             w->st);
      BIPB_LAUNCHED(s);
    }
    k_sumsq<<<w->nblk, kBS, 0, s->stream>>>(len, w->w.p, w->part.p, w->st, 0);
    BIPB_LAUNCHED(s);
    k_normalize<<<w->nblk, kBS, 0, s->stream>>>(len, j, m1, w->nblk, w->w.p, vj + len, w->part.p, w->H.p,
                                                 w->st, 0);
    BIPB_LAUNCHED(s);
    k_givens<<<1, 1, 0, s->stream>>>(j, m1, w->H.p, w->cs.p, w->sn.p, w->g.p, w->st);
    BIPB_LAUNCHED(s);
  }
  k_lsq<<<1, 1, 0, s->stream>>>(m1, w->H.p, w->cs.p, w->sn.p, w->g.p, w->y.p, w->z.p, w->st);
  BIPB_LAUNCHED(s);
  k_update<<<w->nblk, kBS, 0, s->stream>>>(len, m1, w->V.p, w->d.p, w->y.p, w->z.p, w->g.p, w->st);
  BIPB_LAUNCHED(s);
  k_next_cycle<<<1, 1, 0, s->stream>>>(m1, w->g.p, w->st);
  BIPB_LAUNCHED(s);
}

void run_cycle(Surface* s, GmresWork* w, const bipb_medium& med, int precision, bool transpose) {
  // A recorded cycle bakes in the medium and every buffer address, so it is
  // tagged with both and re-recorded when either changes.
  const int key = precision * 2 + (transpose ? 1 : 0);
  const GraphTag tag{s->alloc_gen, med.eps_in, med.eps_out, med.kappa};
  auto it = w->graphs.find(key);
  if (it != w->graphs.end() && it->second.tag == tag && it->second.events.empty() == !s->timer.on) {
    BIPB_CUDA(cudaGraphLaunch(it->second.exec, s->stream));
    s->launches += it->second.kernels;
    w->replayed = &it->second.events;
    return;
  }
  // a plain launch first: it runs this cycle and creates every scratch buffer
  issue_cycle(s, w, med, precision, transpose);
  const GraphTag after{s->alloc_gen, med.eps_in, med.eps_out, med.kappa};
  // record a copy of the cycle for the next calls (the capture does not run it)
  cudaGraph_t graph = nullptr;
  std::vector<EventPair> evs;
  BIPB_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  s->timer.capture = &evs;
  s->recording = true;
  s->recorded_launches = 0;
  try {
    issue_cycle(s, w, med, precision, transpose);
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
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  BIPB_CUDA(e);
  if (it != w->graphs.end()) {
    cudaGraphExecDestroy(it->second.exec);
    for (auto& e : it->second.events) s->timer.pool.push_back(e.a), s->timer.pool.push_back(e.b);
  }
  w->graphs[key] = Recorded{exec, after, std::move(evs), kernels};
}

DevState read_state(Surface* s, GmresWork* w) {
  BIPB_CUDA(cudaMemcpyAsync(w->st_host, w->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  if (s->timer.on) {
    s->timer.collect();
    if (w->replayed)
      for (auto& e : *w->replayed) s->timer.add(e);
  }
  w->replayed = nullptr;
  return *w->st_host;
}

// GMRES on op(A) d = r0 (d starts at zero).  Returns iterations used.
// Stops at recurrence estimate <= tol (relative to ||r0||) or max_iter.
int gmres_core(Surface* s, GmresWork* w, const bipb_medium& med, int precision, bool transpose,
               const double* r0, double tol, int max_iter, DevState* out) {
  const int len = (int)(2 * s->n);
  BIPB_CUDA(cudaMemsetAsync(w->d.p, 0, (size_t)len * sizeof(double), s->stream));
  k_init_state<<<1, 1, 0, s->stream>>>(w->st, w->m, max_iter, tol);
  BIPB_LAUNCHED(s);
  start_cycle(s, w, r0, true);
  DevState h = read_state(s, w);
  while (!h.conv && !h.stop) {
    run_cycle(s, w, med, precision, transpose);
    h = read_state(s, w);
  }
  *out = h;
  return h.iters;
}

double norm2(Surface* s, GmresWork* w, const double* v) {
  const int len = (int)(2 * s->n);
  k_sumsq<<<w->nblk, kBS, 0, s->stream>>>(len, v, w->part.p, w->st, 1);
  BIPB_LAUNCHED(s);
  std::vector<double> h(w->nblk);
  BIPB_CUDA(cudaMemcpyAsync(h.data(), w->part.p, w->nblk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BIPB_CUDA(cudaStreamSynchronize(s->stream));
  double acc = 0.0;
  for (double v2 : h) acc += v2;
  return std::sqrt(acc);
}

}  // namespace

SolveResult gmres_solve(Surface* s, const bipb_medium& med, const bipb_solve_params& p, bool transpose,
                        const double* rhs, double* x, bool warm) {
  SolveResult res;
  const int m = p.restart > 0 ? p.restart : 10;
  const int max_iter = p.max_iter > 0 ? p.max_iter : 1000;
  GmresWork* w = workspace(s, m);
  const int len = (int)(2 * s->n);
  const int nb = blocks(len);
  const double bnorm = norm2(s, w, rhs);
  if (bnorm == 0.0) {
    BIPB_CUDA(cudaMemsetAsync(x, 0, (size_t)len * sizeof(double), s->stream));
    res.converged = 1;
    return res;
  }
  // r = rhs - A x (or rhs when starting from zero)
  if (warm) {
    matvec(s, med, BIPB_FP64, transpose, x, w->t.p, nullptr);
    res.matvecs64++;
    k_sub<<<nb, kBS, 0, s->stream>>>(len, rhs, w->t.p, w->r.p);
  } else {
    BIPB_CUDA(cudaMemsetAsync(x, 0, (size_t)len * sizeof(double), s->stream));
    BIPB_CUDA(cudaMemcpyAsync(w->r.p, rhs, (size_t)len * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  }
  BIPB_LAUNCHED(s);
  double rel = warm ? norm2(s, w, w->r.p) / bnorm : 1.0;
  const bool mixed = p.precision == BIPB_MIXED;
  const double inner_floor = p.inner_tol > 0 ? p.inner_tol : 1e-6;
  const int inner_cap = p.inner_max_iter > 0 ? p.inner_max_iter : 200;
  int iters = 0;
  while (rel > p.tol && iters < max_iter) {
    double tol_rel;
    int cap = max_iter - iters;
    if (mixed) {
      tol_rel = std::max(inner_floor, 0.3 * p.tol / rel);
      cap = std::min(cap, inner_cap);
    } else {
      tol_rel = p.tol / rel;
    }
    DevState h;
    int used = gmres_core(s, w, med, mixed ? BIPB_FP32 : BIPB_FP64, transpose, w->r.p, tol_rel, cap, &h);
    iters += used;
    if (mixed) {
      res.matvecs32 += used;
      res.refine_steps++;
    } else {
      res.matvecs64 += used;
    }
    // x += d ; r = rhs - A x (FP64)
    k_axpy<<<nb, kBS, 0, s->stream>>>(len, 1.0, w->d.p, x);
    BIPB_LAUNCHED(s);
    matvec(s, med, BIPB_FP64, transpose, x, w->t.p, nullptr);
    res.matvecs64++;
    k_sub<<<nb, kBS, 0, s->stream>>>(len, rhs, w->t.p, w->r.p);
    BIPB_LAUNCHED(s);
    double new_rel = norm2(s, w, w->r.p) / bnorm;
    if (!mixed && !h.conv) {  // hit the iteration cap
      rel = new_rel;
      break;
    }
    if (mixed && res.refine_steps >= 3 && new_rel > 0.1 * rel) {  // refinement stalled
      rel = new_rel;
      break;
    }
    rel = new_rel;
  }
  res.iters = iters;
  res.rel_residual = rel;
  res.converged = rel <= p.tol ? 1 : 0;
  return res;
}

}  // namespace bipb
