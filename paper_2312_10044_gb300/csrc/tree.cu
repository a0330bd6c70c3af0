// Far-field (treecode) FP32 mat-vec of Eqs. 5-6, after Sec. 2.2.3.
//
// The mat-vec is an N-body sum per target over sources carrying
// a_j = ds_j psi_j and m_j = ds_j phi_j n_j (K2 and K4 are linear in the
// source normal, so m_j carries it).  The transpose A^T w is the same kind of
// sum: output element t gathers column t of A, whose entries of row element
// j depend on n_j only through K3 and K4, linearly, so the sources carry
// a_j = wphi_j and m_j = wpsi_j n_j, the pair is the transposed one
// (pair_transpose, pair.cuh) and the output element's area multiplies the
// sums.  The tree, the lists and the proxies serve both directions.  The elements form a binary tree of
// clusters; a cluster holding more than `leaf` elements is split in two at
// the median of its longest box side (ties by element index), so every
// cluster is one range of element positions in tree order.  Targets are
// taken leaf by leaf: for target leaf B a cluster c is far when
//   r_c + theta r_B <= theta |x_B - x_c|
// (box centres, half box diagonals), which implies the paper's acceptance
// criterion r_c / |x - x_c| <= theta for every target of B.  Traversal from
// the root gives each leaf a list of source ranges:
//   far c with more elements than proxies -> the (p+1)^3 proxy sources of c,
//   far c otherwise, or a near leaf       -> c's elements (summed directly),
//   a near cluster                        -> its two children.
// A proxy source sits at a Chebyshev point s_k of c's box and carries
//   a_k = sum_{j in c} L_k(x_j) a_j,   m_k = sum_{j in c} L_k(x_j) m_j
// with L_k the tensor-product Lagrange basis of degree p per coordinate
// (barycentric form): a degree-p polynomial in the source position stands in
// for the kernel over a far cluster, as the Taylor series about the cluster
// centre does in the paper.  Because proxies and elements are records of the
// same form (position, a, m), every list entry is summed by the one ordered
// pair formula (pair_forward, pair.cuh) and the far-field pass has the shape
// of the direct pass.
//
// One mat-vec is five launches on the handle's stream:
//   k_tree_pack   element records in tree order (gathered through perm);
//   k_tree_up     partial proxy weights, one CTA per piece of <= 2048
//                 elements of a far cluster (FP32 per 32 elements, FP64 across);
//   k_tree_proxy  proxy records (pieces added in order, FP64);
//   k_tree_far    one CTA per work item: a target leaf (one target per thread)
//                 against a run of its list's records, streamed through shared
//                 memory; FP32 partial sums per item;
//   k_tree_reduce per target, its leaf's items in order (FP64), 1/(4 pi) and
//                 the diagonal, scattered back to element order.
// Every sum is in a fixed order, so the pass is bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.cuh"

namespace bipb {

namespace {

constexpr double kInv4PiT = 1.0 / (4.0 * kPi);
constexpr int kUpPiece = 2048;  // elements per piece of the upward pass
constexpr int kUpChunk = 32;    // elements staged per step of the upward pass
constexpr int kFarCH = 256;     // records per shared-memory chunk of the far-field kernel
constexpr int kMaxLeaf = 512;

__device__ __forceinline__ bool tree_skipped(const int* skip, int stride, int sys) {
  return skip != nullptr && skip[(size_t)sys * stride] != 0;
}

// ------------------------------------------------------------------ kernels
// rec[k][t] = (x, a = ds psi), (m = ds phi n, 0) of element perm[t], system k;
// transposed: (x, a = wphi), (m = wpsi n, 0)
__global__ void k_tree_pack(int n, int rec_stride, bool transpose, const int* __restrict__ perm,
                            const double4_32a* __restrict__ tgt64, const int4* __restrict__ lay,
                            const double* __restrict__ u, float4* __restrict__ rec, const int* __restrict__ skip,
                            int skip_stride) {
  const int k = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || tree_skipped(skip, skip_stride, k)) return;
  const int4 L = lay[k];
  const int e = perm[t];
  const double4_32a g = tgt64[2 * (L.x + e)], v = tgt64[2 * (L.x + e) + 1];
  const double phi = u[L.z + e], psi = u[L.z + L.y + e];
  const double a = transpose ? phi : g.w * psi, f = transpose ? psi : g.w * phi;
  const size_t o = 2 * ((size_t)k * rec_stride + t);
  rec[o] = make_float4((float)g.x, (float)g.y, (float)g.z, (float)a);
  rec[o + 1] = make_float4((float)(f * v.x), (float)(f * v.y), (float)(f * v.z), 0.f);
}

// Partial proxy weights of one piece of a far cluster: for proxy q = (q0, q1, q2),
//   upart[.][q] = sum over the piece's elements of l_q0(x) l_q1(y) l_q2(z) (a, m),
// with l_i the barycentric Lagrange basis at the cluster's Chebyshev nodes
// (weights (-1)^i, halved at both ends).  An element on a node takes the
// node's basis value 1 exactly.
template <int DEG>
__global__ void __launch_bounds__(256) k_tree_up(const int4* __restrict__ pieces, const float* __restrict__ nodes,
                                                 int rec_stride, const float4* __restrict__ rec,
                                                 double* __restrict__ upart, int n_pieces,
                                                 const int* __restrict__ skip, int skip_stride) {
  constexpr int NP = DEG + 1, P = NP * NP * NP, PT = (P + 255) / 256;
  __shared__ float bas[kUpChunk][3][NP];
  __shared__ float4 val[kUpChunk];
  __shared__ float nd[3][NP];
  const int k = blockIdx.y;
  if (tree_skipped(skip, skip_stride, k)) return;
  const int4 pc = pieces[blockIdx.x];  // {slot, first position, count, 0}
  if (threadIdx.x < 3 * NP) nd[threadIdx.x / NP][threadIdx.x % NP] = nodes[(size_t)pc.x * 3 * NP + threadIdx.x];
  double acc[PT][4];
#pragma unroll
  for (int r = 0; r < PT; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.0;
  const float4* R = rec + 2 * (size_t)k * rec_stride;
  for (int c0 = 0; c0 < pc.z; c0 += kUpChunk) {
    const int cnt = min(kUpChunk, pc.z - c0);
    __syncthreads();  // nodes staged; the previous chunk consumed
    const int q = threadIdx.x;
    if (q < 3 * cnt) {  // basis values of element q / 3 along coordinate q % 3
      const int e = q / 3, d = q % 3;
      const float4 r0 = R[2 * (size_t)(pc.y + c0 + e)];
      const float t = d == 0 ? r0.x : (d == 1 ? r0.y : r0.z);
      float w[NP];
      float sum = 0.f;
      int hit = -1;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const float diff = t - nd[d][i];
        const float wi = ((i & 1) ? -1.f : 1.f) * ((i == 0 || i == DEG) ? 0.5f : 1.f);
        if (fabsf(diff) < 1e-30f) hit = i;
        w[i] = wi / diff;
        sum += w[i];
      }
      const float inv = 1.f / sum;
#pragma unroll
      for (int i = 0; i < NP; ++i) bas[e][d][i] = hit >= 0 ? (i == hit ? 1.f : 0.f) : w[i] * inv;
    } else if (q >= 128 && q < 128 + cnt) {
      const int e = q - 128;
      const size_t o = 2 * (size_t)(pc.y + c0 + e);
      const float4 r0 = R[o], r1 = R[o + 1];
      val[e] = make_float4(r0.w, r1.x, r1.y, r1.z);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int kp = threadIdx.x + 256 * r;
      if (kp >= P) continue;
      const int k0 = kp / (NP * NP), k1 = (kp / NP) % NP, k2 = kp % NP;
      float sa = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
      for (int e = 0; e < cnt; ++e) {
        const float w = bas[e][0][k0] * bas[e][1][k1] * bas[e][2][k2];
        const float4 v = val[e];
        sa = fmaf(w, v.x, sa);
        sx = fmaf(w, v.y, sx);
        sy = fmaf(w, v.z, sy);
        sz = fmaf(w, v.w, sz);
      }
      acc[r][0] += sa, acc[r][1] += sx, acc[r][2] += sy, acc[r][3] += sz;
    }
  }
#pragma unroll
  for (int r = 0; r < PT; ++r) {
    const int kp = threadIdx.x + 256 * r;
    if (kp >= P) continue;
    double* o = upart + 4 * ((size_t)(k * n_pieces + blockIdx.x) * P + kp);
    o[0] = acc[r][0], o[1] = acc[r][1], o[2] = acc[r][2], o[3] = acc[r][3];
  }
}

// Proxy records after the element records: (s_q, a_q), (m_q, 0), the pieces
// of the slot's cluster added in order.
template <int DEG>
__global__ void k_tree_proxy(int n_slots, const int2* __restrict__ up_tab, const float* __restrict__ nodes,
                             const double* __restrict__ upart, int n_pieces, int n, int rec_stride,
                             float4* __restrict__ rec, const int* __restrict__ skip, int skip_stride) {
  constexpr int NP = DEG + 1, P = NP * NP * NP;
  const int k = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_slots * P || tree_skipped(skip, skip_stride, k)) return;
  const int slot = idx / P, kp = idx % P;
  const int k0 = kp / (NP * NP), k1 = (kp / NP) % NP, k2 = kp % NP;
  const int2 T = up_tab[slot];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = T.x; p < T.x + T.y; ++p) {
    const double* v = upart + 4 * ((size_t)(k * n_pieces + p) * P + kp);
    s[0] += v[0], s[1] += v[1], s[2] += v[2], s[3] += v[3];
  }
  const float* nd = nodes + (size_t)slot * 3 * NP;
  const size_t o = 2 * ((size_t)k * rec_stride + n + idx);
  rec[o] = make_float4(nd[k0], nd[NP + k1], nd[2 * NP + k2], (float)s[0]);
  rec[o + 1] = make_float4((float)s[1], (float)s[2], (float)s[3], 0.f);
}

// The ordered pair of the far-field pass: A u (pair_forward: accP, accQ the
// phi and psi rows) or A^T w (pair_transpose: the phi and psi outputs).
template <bool TRANS, bool MASK>
__device__ __forceinline__ void tree_pair(const float4& g, const float4& v, const float4& A, const float4& B, bool self,
                                          const PairConst<float>& c, float& accP, float& accQ) {
  if (TRANS)
    pair_transpose<MASK>(g.x, g.y, g.z, v.x, v.y, v.z, A.x, A.y, A.z, A.w, B.x, B.y, B.z, self, c, accP, accQ);
  else
    pair_forward<MASK>(g.x, g.y, g.z, v.x, v.y, v.z, A.x, A.y, A.z, A.w, B.x, B.y, B.z, self, c, accP, accQ);
}

// One work item: the targets of one leaf (thread t: position lf.x + t) against
// the records of segments [it.y, it.z).  The self pair is masked in the
// segments that overlap the leaf's own positions.
template <bool TRANS>
__global__ void __launch_bounds__(kMaxLeaf) k_tree_far(const int4* __restrict__ items, const int2* __restrict__ segs,
                                                      const int4* __restrict__ leaf_tab, const int* __restrict__ perm,
                                                      const float4* __restrict__ tgt32,
                                                      const float4* __restrict__ rec, int rec_stride,
                                                      float* __restrict__ part, int n_items, int lmax,
                                                      PairConst<float> c, const int* __restrict__ skip,
                                                      int skip_stride) {
  __shared__ float4 sh[2 * kFarCH];
  const int k = blockIdx.y;
  if (tree_skipped(skip, skip_stride, k)) return;
  const int4 it = items[blockIdx.x];
  const int4 lf = leaf_tab[it.x];
  const int t = threadIdx.x;
  const bool active = t < lf.y;
  const int pos = lf.x + min(t, lf.y - 1);
  const int e = perm[pos];
  const float4 g = tgt32[2 * (size_t)e], v = tgt32[2 * (size_t)e + 1];
  float accP = 0.f, accQ = 0.f;
  const float4* R = rec + 2 * (size_t)k * rec_stride;
  for (int sg = it.y; sg < it.z; ++sg) {
    const int2 S = segs[sg];
    const bool self = S.x < lf.x + lf.y && S.x + S.y > lf.x;
    for (int j0 = 0; j0 < S.y; j0 += kFarCH) {
      const int m = min(kFarCH, S.y - j0);
      __syncthreads();
      const float4* src = R + 2 * (size_t)(S.x + j0);
      for (int q = t; q < 2 * m; q += blockDim.x) sh[q] = src[q];
      __syncthreads();
      if (!active) continue;
      if (!self) {
        if (m == kFarCH) {
#pragma unroll 8
          for (int jj = 0; jj < kFarCH; ++jj) tree_pair<TRANS, false>(g, v, sh[2 * jj], sh[2 * jj + 1], false, c, accP, accQ);
        } else {
          for (int jj = 0; jj < m; ++jj) tree_pair<TRANS, false>(g, v, sh[2 * jj], sh[2 * jj + 1], false, c, accP, accQ);
        }
      } else {
        for (int jj = 0; jj < m; ++jj)
          tree_pair<TRANS, true>(g, v, sh[2 * jj], sh[2 * jj + 1], S.x + j0 + jj == pos, c, accP, accQ);
      }
    }
  }
  if (active) {
    float* o = part + 2 * (size_t)lmax * ((size_t)k * n_items + blockIdx.x);
    o[t] = accP;
    o[lmax + t] = accQ;
  }
}

// y of element perm[t]: diag u - 1/(4 pi) (sum over the leaf's items in order),
// the sum times the element's area for the transpose
__global__ void k_tree_reduce(int n, const int* __restrict__ perm, const int* __restrict__ leaf_of,
                              const int4* __restrict__ leaf_tab, const float* __restrict__ part, int n_items,
                              int lmax, const int4* __restrict__ lay, const double4_32a* __restrict__ area_of,
                              const double* __restrict__ u, double* __restrict__ y, double dphi, double dpsi,
                              const int* __restrict__ skip, int skip_stride) {
  const int k = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || tree_skipped(skip, skip_stride, k)) return;
  const int4 lf = leaf_tab[leaf_of[t]];
  const int local = t - lf.x;
  double sp = 0.0, sq = 0.0;
  for (int i = lf.z; i < lf.z + lf.w; ++i) {
    const float* o = part + 2 * (size_t)lmax * ((size_t)k * n_items + i);
    sp += (double)o[local];
    sq += (double)o[lmax + local];
  }
  const int4 L = lay[k];
  const int e = perm[t];
  const double w = area_of != nullptr ? area_of[2 * (L.x + e)].w * kInv4PiT : kInv4PiT;
  y[L.z + e] = dphi * u[L.z + e] - w * sp;
  y[L.z + L.y + e] = dpsi * u[L.z + L.y + e] - w * sq;
}

// ------------------------------------------------------------------ host: tree and lists
struct Node {
  int start, end;
  double lo[3], hi[3];
  int left, right;
};

// The tree of clusters over the centroids as given (FP64), in the order the
// definition above fixes (median split of the longest side, ties by index).
void build_nodes(const double* x, int n, int leaf, std::vector<int>& perm, std::vector<Node>& nodes) {
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  nodes.clear();
  auto make = [&](int s, int e) {
    Node nd;
    nd.start = s, nd.end = e, nd.left = nd.right = -1;
    for (int d = 0; d < 3; ++d) nd.lo[d] = INFINITY, nd.hi[d] = -INFINITY;
    for (int i = s; i < e; ++i)
      for (int d = 0; d < 3; ++d) {
        const double v = x[3 * (size_t)perm[i] + d];
        nd.lo[d] = std::min(nd.lo[d], v);
        nd.hi[d] = std::max(nd.hi[d], v);
      }
    nodes.push_back(nd);
    return (int)nodes.size() - 1;
  };
  std::vector<int> stack{make(0, n)};
  while (!stack.empty()) {
    const int k = stack.back();
    stack.pop_back();
    const Node nd = nodes[k];
    const int cnt = nd.end - nd.start;
    if (cnt <= leaf) continue;
    int d = 0;
    for (int q = 1; q < 3; ++q)
      if (nd.hi[q] - nd.lo[q] > nd.hi[d] - nd.lo[d]) d = q;
    std::sort(perm.begin() + nd.start, perm.begin() + nd.end, [&](int a, int b) {
      const double xa = x[3 * (size_t)a + d], xb = x[3 * (size_t)b + d];
      return xa < xb || (xa == xb && a < b);
    });
    const int h = cnt / 2;
    const int l = make(nd.start, nd.start + h);
    const int r = make(nd.start + h, nd.end);
    nodes[k].left = l;
    nodes[k].right = r;
    stack.push_back(r);
    stack.push_back(l);
  }
}

void centre_radius(const Node& nd, double c[3], double* r) {
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    c[d] = 0.5 * (nd.lo[d] + nd.hi[d]);
    const double h = 0.5 * (nd.hi[d] - nd.lo[d]);
    s = s + h * h;
  }
  *r = std::sqrt(s);
}

struct Entry {
  bool far;
  int a, b;  // direct: positions [a, b); far: node a
};

void collect(const std::vector<Node>& nodes, int k, const double xb[3], double rb, double theta, int n_proxy,
             std::vector<Entry>& out) {
  const Node& nd = nodes[k];
  double xc[3], rc;
  centre_radius(nd, xc, &rc);
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double dd = xb[d] - xc[d];
    s = s + dd * dd;
  }
  const double dist = std::sqrt(s);
  const int count = nd.end - nd.start;
  if (rc + theta * rb <= theta * dist) {
    if (count > n_proxy)
      out.push_back(Entry{true, k, 0});
    else
      out.push_back(Entry{false, nd.start, nd.end});
  } else if (nd.left < 0) {
    out.push_back(Entry{false, nd.start, nd.end});
  } else {
    collect(nodes, nd.left, xb, rb, theta, n_proxy, out);
    collect(nodes, nd.right, xb, rb, theta, n_proxy, out);
  }
}

template <int DEG>
void launch_up(const FarField* f, cudaStream_t st, int K, const int* skip, int skip_stride) {
  k_tree_up<DEG><<<dim3(f->n_up, K), 256, 0, st>>>(f->up_pieces.p, f->nodes.p, f->rec_stride, f->rec.p, f->upart.p,
                                                    f->n_up, skip, skip_stride);
}
template <int DEG>
void launch_proxy(const FarField* f, cudaStream_t st, int K, const int* skip, int skip_stride) {
  constexpr int P = (DEG + 1) * (DEG + 1) * (DEG + 1);
  k_tree_proxy<DEG><<<dim3((f->n_slots * P + 255) / 256, K), 256, 0, st>>>(
      f->n_slots, f->up_tab.p, f->nodes.p, f->upart.p, f->n_up, f->n, f->rec_stride, f->rec.p, skip, skip_stride);
}

int far_occupancy(int nt) {  // both directions have the same shape; the forward kernel sets the plan
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tree_far<false>, nt, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    o = 1;
  }
  return std::max(o, 1);
}

std::unique_ptr<FarField> build_far_field(Surface* s) {
  auto f = std::make_unique<FarField>();
  f->theta = s->far_theta;
  f->degree = s->far_degree;
  f->leaf = s->far_leaf;
  const int n = (int)s->n;
  f->n = n;
  const int np1 = f->degree + 1, P = np1 * np1 * np1;
  std::vector<int> perm;
  std::vector<Node> nodes;
  build_nodes(s->raw_centroids.data(), n, f->leaf, perm, nodes);
  // leaves in tree order
  std::vector<int> leaves;
  for (int k = 0; k < (int)nodes.size(); ++k)
    if (nodes[k].left < 0) leaves.push_back(k);
  std::sort(leaves.begin(), leaves.end(), [&](int a, int b) { return nodes[a].start < nodes[b].start; });
  f->n_leaves = (int)leaves.size();
  // interaction lists (adjacent direct ranges merged)
  std::vector<std::vector<Entry>> lists(leaves.size());
  std::vector<int> slot_of(nodes.size(), -1);
  for (size_t li = 0; li < leaves.size(); ++li) {
    double xb[3], rb;
    centre_radius(nodes[leaves[li]], xb, &rb);
    std::vector<Entry> raw;
    collect(nodes, 0, xb, rb, f->theta, P, raw);
    auto& out = lists[li];
    for (const Entry& e : raw) {
      if (!e.far && !out.empty() && !out.back().far && out.back().b == e.a)
        out.back().b = e.b;
      else
        out.push_back(e);
      if (e.far) slot_of[e.a] = 0;
    }
  }
  std::vector<int> slot_node;
  for (int k = 0; k < (int)nodes.size(); ++k)
    if (slot_of[k] >= 0) slot_of[k] = (int)slot_node.size(), slot_node.push_back(k);
  f->n_slots = (int)slot_node.size();
  f->rec_stride = n + f->n_slots * P;
  // segments of every leaf as record ranges, and their lengths
  std::vector<std::vector<int2>> lseg(leaves.size());
  std::vector<int64_t> lrec(leaves.size(), 0);
  int lmax = 1;
  for (size_t li = 0; li < leaves.size(); ++li) {
    lmax = std::max(lmax, nodes[leaves[li]].end - nodes[leaves[li]].start);
    for (const Entry& e : lists[li]) {
      const int2 sg = e.far ? make_int2(n + slot_of[e.a] * P, P) : make_int2(e.a, e.b - e.a);
      lseg[li].push_back(sg);
      lrec[li] += sg.y;
    }
  }
  f->lmax = lmax;
  f->nt = (lmax + 31) / 32 * 32;
  // cut every leaf's list into pieces of about L records; L keeps whole waves busy
  const int slots = s->num_sms * far_occupancy(f->nt);
  int64_t rmax = 1;
  for (auto r : lrec) rmax = std::max(rmax, r);
  auto n_items_for = [&](int64_t L) {
    int64_t c = 0;
    for (auto r : lrec) c += std::max<int64_t>(1, (r + L - 1) / L);
    return c;
  };
  int64_t bestL = rmax;
  double best = 1e300;
  for (int64_t L = 256; L < 2 * rmax; L = L + std::max<int64_t>(64, L / 16)) {
    const int64_t c = n_items_for(L);
    const double est = (double)((c + slots - 1) / slots) * (double)(std::min(L, rmax) + 256);
    if (est < best) best = est, bestL = L;
  }
  std::vector<int4> items, leaf_tab(leaves.size());
  std::vector<int2> segs;
  std::vector<int> leaf_of(n);
  f->pair_evals = 0;
  for (size_t li = 0; li < leaves.size(); ++li) {
    const Node& nd = nodes[leaves[li]];
    const int cnt = nd.end - nd.start;
    for (int p = nd.start; p < nd.end; ++p) leaf_of[p] = (int)li;
    f->pair_evals += (int64_t)cnt * lrec[li];
    const int64_t R = lrec[li];
    const int pieces = (int)std::max<int64_t>(1, (R + bestL - 1) / bestL);
    leaf_tab[li] = make_int4(nd.start, cnt, (int)items.size(), pieces);
    // walk the segments, cutting at q_p = p R / pieces
    size_t si = 0;
    int off = 0;  // records of segment si already given out
    for (int p = 0; p < pieces; ++p) {
      int64_t want = (int64_t)(p + 1) * R / pieces - (int64_t)p * R / pieces;
      const int first = (int)segs.size();
      while (want > 0 && si < lseg[li].size()) {
        const int2 sg = lseg[li][si];
        const int take = (int)std::min<int64_t>(want, sg.y - off);
        segs.push_back(make_int2(sg.x + off, take));
        want -= take;
        off += take;
        if (off == sg.y) ++si, off = 0;
      }
      items.push_back(make_int4((int)li, first, (int)segs.size(), 0));
    }
  }
  f->n_items = (int)items.size();
  // upward pieces and Chebyshev nodes of every far cluster (centred, FP32)
  std::vector<int4> up;
  std::vector<int2> up_tab(f->n_slots);
  std::vector<float> nd32((size_t)f->n_slots * 3 * np1);
  const double* ctr = &s->part_center[0];
  for (int sl = 0; sl < f->n_slots; ++sl) {
    const Node& nd = nodes[slot_node[sl]];
    up_tab[sl] = make_int2((int)up.size(), 0);
    for (int p = nd.start; p < nd.end; p += kUpPiece) up.push_back(make_int4(sl, p, std::min(kUpPiece, nd.end - p), 0));
    up_tab[sl].y = (int)up.size() - up_tab[sl].x;
    double ext[3], emax = 0.0;
    for (int d = 0; d < 3; ++d) ext[d] = nd.hi[d] - nd.lo[d], emax = std::max(emax, ext[d]);
    for (int d = 0; d < 3; ++d) {
      const double e = std::max(ext[d], 1e-3 * emax);
      const double c = 0.5 * (nd.lo[d] + nd.hi[d]);
      for (int i = 0; i <= f->degree; ++i)
        nd32[((size_t)sl * 3 + d) * np1 + i] = (float)(c + (0.5 * e) * std::cos(kPi * i / f->degree) - ctr[d]);
    }
  }
  f->n_up = (int)up.size();
  // device copies
  cudaStream_t st = s->stream;
  auto put = [&](auto& buf, const auto& v) {
    using T = typename std::decay_t<decltype(v)>::value_type;
    buf.ensure(std::max<size_t>(v.size(), 1), st);
    if (!v.empty())
      BIPB_CUDA(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  };
  put(f->perm, perm);
  put(f->leaf_of, leaf_of);
  put(f->leaf_tab, leaf_tab);
  put(f->items, items);
  put(f->segs, segs);
  put(f->up_pieces, up);
  put(f->up_tab, up_tab);
  put(f->nodes, nd32);
  BIPB_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
  ++s->alloc_gen;
  return f;
}

}  // namespace

FarField* far_field(Surface* s) {
  BIPB_REQUIRE(!s->batch, "the far-field mat-vec needs a single-surface handle");
  FarField* f = s->far.get();
  if (f && f->theta == s->far_theta && f->degree == s->far_degree && f->leaf == s->far_leaf) return f;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BIPB_CUDA(cudaStreamIsCapturing(s->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) throw Error(BIPB_ERR_CUDA, "far-field tree built while recording a graph");
  s->far = build_far_field(s);
  return s->far.get();
}

void matvec_tree(Surface* s, const SysLayout& L, const PairConst<float>& c, bool transpose, const double* u, double* y,
                 double dphi, double dpsi, const int* skip, int skip_stride) {
  for (int k = 0; k < L.K; ++k)
    BIPB_REQUIRE(L.geo_off[k] == 0 && L.n[k] == (int)s->n, "the far-field mat-vec covers one surface");
  FarField* f = far_field(s);
  const int K = L.K;
  const int P = (f->degree + 1) * (f->degree + 1) * (f->degree + 1);
  if (f->rec.ensure(2 * (size_t)f->rec_stride * K, s->stream)) ++s->alloc_gen;
  if (f->part.ensure(2 * (size_t)f->lmax * f->n_items * K, s->stream)) ++s->alloc_gen;
  if (f->upart.ensure(std::max<size_t>(1, 4 * (size_t)P * f->n_up * K), s->stream)) ++s->alloc_gen;
  const int4* lay = s->lay_dev(L);
  const int nb = (f->n + 255) / 256;
  k_tree_pack<<<dim3(nb, K), 256, 0, s->stream>>>(f->n, f->rec_stride, transpose, f->perm.p, s->tgt64.p, lay, u,
                                                  f->rec.p, skip, skip_stride);
  BIPB_LAUNCHED(s);
  if (f->n_up > 0) {
    switch (f->degree) {
      case 4: launch_up<4>(f, s->stream, K, skip, skip_stride); break;
      case 6: launch_up<6>(f, s->stream, K, skip, skip_stride); break;
      default: launch_up<8>(f, s->stream, K, skip, skip_stride); break;
    }
    BIPB_LAUNCHED(s);
    switch (f->degree) {
      case 4: launch_proxy<4>(f, s->stream, K, skip, skip_stride); break;
      case 6: launch_proxy<6>(f, s->stream, K, skip, skip_stride); break;
      default: launch_proxy<8>(f, s->stream, K, skip, skip_stride); break;
    }
    BIPB_LAUNCHED(s);
  }
  {
    TimedLaunch tl(s, kTMvTree);
    if (transpose)
      k_tree_far<true><<<dim3(f->n_items, K), f->nt, 0, s->stream>>>(f->items.p, f->segs.p, f->leaf_tab.p,
                                                                    f->perm.p, s->tgt32.p, f->rec.p, f->rec_stride,
                                                                    f->part.p, f->n_items, f->lmax, c, skip,
                                                                    skip_stride);
    else
      k_tree_far<false><<<dim3(f->n_items, K), f->nt, 0, s->stream>>>(f->items.p, f->segs.p, f->leaf_tab.p,
                                                                     f->perm.p, s->tgt32.p, f->rec.p, f->rec_stride,
                                                                     f->part.p, f->n_items, f->lmax, c, skip,
                                                                     skip_stride);
    BIPB_LAUNCHED(s);
  }
  k_tree_reduce<<<dim3(nb, K), 256, 0, s->stream>>>(f->n, f->perm.p, f->leaf_of.p, f->leaf_tab.p, f->part.p,
                                                    f->n_items, f->lmax, lay, transpose ? s->tgt64.p : nullptr, u, y,
                                                    dphi, dpsi, skip, skip_stride);
  BIPB_LAUNCHED(s);
}

}  // namespace bipb
