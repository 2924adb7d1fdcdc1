// Path refinement (Section 2.3): gradient descent on the path length (Eq. 2) with
// re-projection of reflection points onto the point cloud, final visibility,
// label-based and first-Fresnel-zone duplicate removal.
//
// B300 design: one thread per coarse path holds the whole path state in FP64
// (positions, bases, the gradient and the final length), because the descent's
// stability needs it; the re-projection ray and its Eq. 1 march run in FP32 in
// the frame of the intersected IE (offsets of a few decimetres), and the final
// visibility rays are the FP32 traversal of the tracer.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nimbus_host.hpp"

namespace nb {

namespace {

constexpr double C_LIGHT = 299792458.0;

struct DRefine {
  double delta, gamma, grad_stop, lambda, hs;
  int rho;
};

struct CoarseView {
  const uint32_t *tx, *rx, *nint, *types, *ie, *lab, *gid;
  int64_t n;
};

__device__ __forceinline__ d3 dunit(d3 a) {
  double n = sqrt(dot(a, a));
  return n > 0.0 ? (1.0 / n) * a : a;
}

// Re-projection (Section 2.3): the ray from P toward the updated point R is
// intersected (Eq. 1 march) with the point IEs of label `label` in the 3x3x3 voxels
// around R; the hit nearest R wins (ties: lower IE index).  Returns the new
// interaction point and the Eq. 1 normal there.
__device__ bool reproject(const DScene& s, d3 P, d3 R, uint32_t label, d3* c_out, d3* n_out) {
  d3 dv = R - P;
  double tR = len(dv);
  if (tR < 1e-12) return false;
  d3 d = (1.0 / tR) * dv;
  float3 df = tof(d);
  int v[3] = {(int)floor((R.x - s.odx) / s.hd), (int)floor((R.y - s.ody) / s.hd), (int)floor((R.z - s.odz) / s.hd)};
  bool found = false;
  double best = 0.0, best_t = 0.0;
  uint32_t best_id = 0;
  unsigned long long bytes = 0;
  const double rs2 = (double)s.r_sub * (double)s.r_sub;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int u0 = v[0] + dx, u1 = v[1] + dy, u2 = v[2] + dz;
        if (!in_grid(s, u0, u1, u2)) continue;
        uint2 cell = __ldg(&s.cells[cell_index(s, u0, u1, u2)]);
        for (uint32_t k = 0; k < cell.y; ++k) {
          uint32_t id = cell.x + k;
          const IERec* r = &s.ies[id];
          float4 nm = __ldg(&r->nrm_meta);
          if ((__float_as_uint(nm.w) & 1u) != IE_POINT) continue;
          if (__float_as_uint(__ldg(&r->rp_lab).w) != label) continue;
          float4 sc = __ldg(&r->sc_pc);
          d3 scd = D3(sc.x, sc.y, sc.z);
          double tc = fmax(dot(scd - P, d), 0.0);
          d3 q = (P + tc * d) - scd;
          if (dot(q, q) > rs2) continue;
          float4 bb = __ldg(&r->bbc_pb);
          d3 c = D3(bb.x, bb.y, bb.z);
          double t0 = dot(c - P, d);
          float3 x0 = tof((P + t0 * d) - c);
          float tau;
          if (!sdf_march(s, __float_as_uint(bb.w), __float_as_uint(sc.w), xyz(bb), x0, df, &tau, bytes)) continue;
          double t = t0 + (double)tau;
          if (!(t > 0.0)) continue;
          double score = fabs(t - tR);
          if (!found || score < best || (score == best && id < best_id)) {
            found = true;
            best = score;
            best_t = t;
            best_id = id;
          }
        }
      }
  if (!found) return false;
  d3 c = P + best_t * d;
  const IERec* r = &s.ies[best_id];
  float4 bb = __ldg(&r->bbc_pb);
  float4 sc = __ldg(&r->sc_pc);
  d3 cb = D3(bb.x, bb.y, bb.z);
  float f;
  float3 n;
  if (!sdf_local(s, __float_as_uint(bb.w), __float_as_uint(sc.w), xyz(bb), tof(c - cb), &f, &n, bytes))
    return false;
  *c_out = c;
  *n_out = D3(n.x, n.y, n.z);
  return true;
}

__global__ void __launch_bounds__(128) k_refine(DScene s, DRefine rp, CoarseView C, const double* txd,
                                                const double* rxd, ExactRec* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * blockDim.x) {
    ExactRec ex;
    const int n = (int)C.nint[i];
    const uint32_t types = C.types[i];
    d3 I[NB_MAXI + 2], c[NB_MAXI + 2], u[NB_MAXI + 2], v[NB_MAXI + 2], w[NB_MAXI + 2], p0[NB_MAXI + 2];
    double tpar[NB_MAXI + 2], elen[NB_MAXI + 2];
    const uint32_t tx = C.tx[i], rx = C.rx[i];
    I[0] = D3(txd[3 * tx], txd[3 * tx + 1], txd[3 * tx + 2]);
    I[n + 1] = D3(rxd[3 * rx], rxd[3 * rx + 1], rxd[3 * rx + 2]);
    ex.tx = tx;
    ex.rx = rx;
    ex.n = (uint32_t)n;
    ex.types = types;
    ex.gid = C.gid[i];
    for (int q = 0; q < NB_MAXI; ++q) {
      ex.lab[q] = C.lab[i * NB_MAXI + q];
      ex.ie[q] = C.ie[i * NB_MAXI + q];
      ex.mat[q] = 255;
      ex.pts[q][0] = ex.pts[q][1] = ex.pts[q][2] = 0.0;
    }
    for (int k = 1; k <= n; ++k) {
      const IERec* r = &s.ies[C.ie[i * NB_MAXI + k - 1]];
      float4 rpl = r->rp_lab, nm = r->nrm_meta;
      ex.mat[k - 1] = (uint8_t)((__float_as_uint(nm.w) >> 8) & 0xffu);
      c[k] = D3(rpl.x, rpl.y, rpl.z);
      I[k] = c[k];
      tpar[k] = 0.0;
      if (!((types >> (k - 1)) & 1u)) {
        onb(dunit(D3(nm.x, nm.y, nm.z)), &u[k], &v[k]);
      } else {
        const double* E = s.edges + 12 * __float_as_uint(r->bbc_pb.w);
        p0[k] = D3(E[0], E[1], E[2]);
        d3 ev = D3(E[3] - E[0], E[4] - E[1], E[5] - E[2]);
        elen[k] = len(ev);
        w[k] = (1.0 / elen[k]) * ev;
      }
    }
    double g[NB_MAXI + 2][2];
    int status = ST_VALID, it = 0;
    bool converged = false;
    double gn = 0.0;
    for (; it < rp.rho; ++it) {
      // gradient of Eq. 2: (e_in + e_out) . (u, v) for reflections, . w for diffractions
      double g2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        d3 e = dunit(I[k] - I[k - 1]) + dunit(I[k] - I[k + 1]);
        if (!((types >> (k - 1)) & 1u)) {
          g[k][0] = dot(e, u[k]);
          g[k][1] = dot(e, v[k]);
        } else {
          g[k][0] = dot(e, w[k]);
          g[k][1] = 0.0;
        }
        g2 += g[k][0] * g[k][0] + g[k][1] * g[k][1];
      }
      gn = sqrt(g2);
      if (gn < rp.grad_stop) {
        converged = true;
        break;
      }
      d3 In[NB_MAXI + 2];
      for (int k = 1; k <= n; ++k) {
        double a = len(I[k] - I[k - 1]), b = len(I[k] - I[k + 1]);
        double eta = rp.gamma / (1.0 / a + 1.0 / b);
        if (!((types >> (k - 1)) & 1u)) {
          double rr = -eta * g[k][0], ss = -eta * g[k][1];
          double l = sqrt(rr * rr + ss * ss);
          if (l > rp.hs) {
            rr *= rp.hs / l;
            ss *= rp.hs / l;
          }
          d3 R = c[k] + rr * u[k] + ss * v[k];     // R_k = c_k + r_k u_k + s_k v_k
          d3 cn, nn;
          if (!reproject(s, I[k - 1], R, ex.lab[k - 1], &cn, &nn)) {
            status = ST_MISS;
            break;
          }
          c[k] = cn;
          onb(dunit(nn), &u[k], &v[k]);
          In[k] = cn;
        } else {
          double dt = -eta * g[k][0];
          if (fabs(dt) > rp.hs) dt = copysign(rp.hs, dt);
          tpar[k] += dt;                            // D_k = c_k + t_k w_k
          In[k] = c[k] + tpar[k] * w[k];
          double along = dot(In[k] - p0[k], w[k]);
          if (along < 0.0 || along > elen[k]) {
            status = ST_OFF_EDGE;
            break;
          }
        }
      }
      if (status != ST_VALID) break;
      for (int k = 1; k <= n; ++k) I[k] = In[k];
    }
    if (status == ST_VALID && !converged) {
      double g2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        d3 e = dunit(I[k] - I[k - 1]) + dunit(I[k] - I[k + 1]);
        double a0 = ((types >> (k - 1)) & 1u) ? dot(e, w[k]) : dot(e, u[k]);
        double a1 = ((types >> (k - 1)) & 1u) ? 0.0 : dot(e, v[k]);
        g2 += a0 * a0 + a1 * a1;
      }
      gn = sqrt(g2);
      if (!(gn < rp.delta)) status = ST_NOT_CONVERGED;
    }
    for (int k = 1; k <= n; ++k) {
      ex.pts[k - 1][0] = I[k].x;
      ex.pts[k - 1][1] = I[k].y;
      ex.pts[k - 1][2] = I[k].z;
    }
    if (status == ST_VALID) {
      // visibility between consecutive path nodes
      unsigned long long bytes = 0;
      for (int k = 0; k <= n && status == ST_VALID; ++k) {
        Endpoint ea{IGN_NONE, NB_NONE_LABEL}, eb{IGN_NONE, NB_NONE_LABEL};
        if (k >= 1) ea = Endpoint{((types >> (k - 1)) & 1u) ? IGN_ANY : IGN_LABEL, ex.lab[k - 1]};
        if (k + 1 <= n) eb = Endpoint{((types >> k) & 1u) ? IGN_ANY : IGN_LABEL, ex.lab[k]};
        if (!visible(s, tof(I[k]), tof(I[k + 1]), ea, eb, bytes)) status = ST_OCCLUDED;
      }
    }
    double L = 0.0;
    for (int k = 0; k <= n; ++k) L += len(I[k + 1] - I[k]);
    ex.length = status == ST_VALID ? L : 0.0;
    ex.delay = ex.length / C_LIGHT;
    ex.grad = gn;
    ex.iters = (uint32_t)it;
    ex.status = (uint32_t)status;
    ex.pad = 0;
    out[i] = ex;
  }
}

// ------------------------------------------------------------ duplicate removal
__global__ void k_best_len(const ExactRec* ex, int64_t n, unsigned long long* best) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (ex[i].status == ST_VALID) atomicMin(&best[ex[i].gid], (unsigned long long)__double_as_longlong(ex[i].length));
}

__global__ void k_best_idx(const ExactRec* ex, int64_t n, const unsigned long long* best, uint32_t* widx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (ex[i].status == ST_VALID &&
        (unsigned long long)__double_as_longlong(ex[i].length) == best[ex[i].gid])
      atomicMin(&widx[ex[i].gid], (uint32_t)i);
}

__global__ void k_winner_flags(const ExactRec* ex, int64_t n, const uint32_t* widx, uint32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (ex[i].status == ST_VALID && widx[ex[i].gid] == (uint32_t)i) ? 1u : 0u;
}

__global__ void k_winner_keys(const ExactRec* ex, const uint32_t* flag, const uint32_t* pos, int64_t n, int n_rx,
                              uint64_t* keys, uint32_t* vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      keys[pos[i]] = (uint64_t)ex[i].tx * (uint64_t)n_rx + ex[i].rx;
      vals[pos[i]] = (uint32_t)i;
    }
}

// Order inside one TX/RX pair: length in micrometre bins (delay order, with ties of
// equal length up to rounding decided by the next keys), interaction types and
// labels, then the IE sequence.
__device__ bool path_less(const ExactRec& a, const ExactRec& b) {
  long long qa = (long long)floor(a.length * 1e6), qb = (long long)floor(b.length * 1e6);
  if (qa != qb) return qa < qb;
  if (a.n != b.n) return a.n < b.n;
  for (uint32_t q = 0; q < a.n; ++q) {
    uint32_t ta = (a.types >> q) & 1u, tb = (b.types >> q) & 1u;
    if (ta != tb) return ta < tb;
    if (a.lab[q] != b.lab[q]) return a.lab[q] < b.lab[q];
  }
  for (uint32_t q = 0; q < a.n; ++q)
    if (a.ie[q] != b.ie[q]) return a.ie[q] < b.ie[q];
  return false;
}

// One thread per TX/RX pair: order its label winners, then drop every path whose
// interaction points all lie in the first Fresnel zones of an earlier kept path
// with the same chain of interaction types.
__global__ void k_fresnel(const ExactRec* ex, const uint64_t* keys, uint32_t* vals, int64_t n, const double* txd,
                          double lambda, uint32_t* keep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i > 0 && keys[i] == keys[i - 1]) continue;   // not the first of its pair
    int64_t e = i;
    while (e < n && keys[e] == keys[i]) ++e;
    for (int64_t a = i + 1; a < e; ++a) {              // insertion sort of the pair
      uint32_t x = vals[a];
      int64_t b = a - 1;
      while (b >= i && path_less(ex[x], ex[vals[b]])) {
        vals[b + 1] = vals[b];
        --b;
      }
      vals[b + 1] = x;
    }
    for (int64_t bI = i; bI < e; ++bI) {
      const ExactRec& B = ex[vals[bI]];
      bool dup = false;
      for (int64_t aI = i; aI < bI && !dup; ++aI) {
        if (!keep[aI]) continue;
        const ExactRec& A = ex[vals[aI]];
        if (A.n != B.n || A.n == 0 || A.types != B.types) continue;
        double px = txd[3 * A.tx], py = txd[3 * A.tx + 1], pz = txd[3 * A.tx + 2];
        double acc = 0.0;
        bool inside = true;
        for (uint32_t q = 0; q < A.n && inside; ++q) {
          double dx = A.pts[q][0] - px, dy = A.pts[q][1] - py, dz = A.pts[q][2] - pz;
          acc += sqrt(dx * dx + dy * dy + dz * dz);
          px = A.pts[q][0]; py = A.pts[q][1]; pz = A.pts[q][2];
          double ak = acc, bk = A.length - acc;
          double r = sqrt(lambda * ak * bk / (ak + bk));
          double ex_ = B.pts[q][0] - A.pts[q][0], ey = B.pts[q][1] - A.pts[q][1], ez = B.pts[q][2] - A.pts[q][2];
          inside = sqrt(ex_ * ex_ + ey * ey + ez * ez) <= r;
        }
        dup = inside;
      }
      keep[bI] = dup ? 0u : 1u;
    }
  }
}

__global__ void k_final(const uint32_t* keep, const uint32_t* pos, const uint32_t* vals, int64_t n, uint32_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (keep[i]) out[pos[i]] = vals[i];
}

unsigned pgrid(int block) {
  static int sms = 0;
  if (!sms) sms = num_sms();
  return (unsigned)(sms * (2048 / block));
}

}  // namespace

int refine_paths(Mem& mem, SceneObj* S, CoarseObj* C, const nimbus_refine_params* p, PathsObj* P, cudaStream_t st) {
  std::string* err = mem.err;
  if (!(p->delta > 0) || p->rho < 0 || !(p->gamma > 0) || !(p->freq_hz > 0)) {
    *err = "refine: invalid parameters";
    return NIMBUS_ERR_ARG;
  }
  P->mem = &mem;
  const int64_t n = C->n;
  P->n_all = n;
  P->counts = C->counts;
  P->counts.n_refined = n;
  NB_TRY(P->own(&P->all, std::max<int64_t>(1, n), st));
  NB_TRY(P->own(&P->final_idx, std::max<int64_t>(1, n), st));
  P->n_final = 0;
  if (n == 0) {
    P->counts.n_paths = 0;
    return NIMBUS_OK;
  }
  DRefine rp;
  rp.delta = p->delta;
  rp.gamma = p->gamma;
  rp.grad_stop = p->grad_stop;
  rp.lambda = C_LIGHT / p->freq_hz;
  rp.hs = S->d.hsd;
  rp.rho = p->rho;
  CoarseView cv{C->tx, C->rx, C->nint, C->types, C->ie, C->lab, C->gid, n};
  const unsigned G = std::min<unsigned>(grid_for(n, 128), pgrid(128));
  k_refine<<<G, 128, 0, st>>>(S->d, rp, cv, C->txd, C->rxd, P->all);
  NB_CUDA(err, cudaGetLastError());
  Scratch sc(&mem, st);
  unsigned long long* best;
  uint32_t *widx, *flag, *pos, *nw, *vals, *vals_alt, *keep, *kpos, *nk;
  uint64_t *keys, *keys_alt;
  const uint32_t ng = C->n_groups_cap;
  NB_TRY(sc.get(&best, ng));
  NB_TRY(sc.get(&widx, ng));
  NB_TRY(sc.get(&flag, n));
  NB_TRY(sc.get(&pos, n));
  NB_TRY(sc.get(&nw, 1));
  NB_CUDA(err, cudaMemsetAsync(best, 0xff, ng * sizeof(unsigned long long), st));
  NB_CUDA(err, cudaMemsetAsync(widx, 0xff, ng * sizeof(uint32_t), st));
  const unsigned G2 = std::min<unsigned>(grid_for(n, 256), pgrid(256));
  k_best_len<<<G2, 256, 0, st>>>(P->all, n, best);
  NB_CUDA(err, cudaGetLastError());
  k_best_idx<<<G2, 256, 0, st>>>(P->all, n, best, widx);
  NB_CUDA(err, cudaGetLastError());
  k_winner_flags<<<G2, 256, 0, st>>>(P->all, n, widx, flag);
  NB_CUDA(err, cudaGetLastError());
  NB_TRY(exclusive_scan(sc, flag, pos, n, nw));
  // valid paths count (for the counters)
  uint32_t hw = 0;
  NB_CUDA(err, cudaMemcpyAsync(&hw, nw, sizeof hw, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t m = hw;
  if (m > 0) {
    NB_TRY(sc.get(&keys, m));
    NB_TRY(sc.get(&keys_alt, m));
    NB_TRY(sc.get(&vals, m));
    NB_TRY(sc.get(&vals_alt, m));
    NB_TRY(sc.get(&keep, m));
    NB_TRY(sc.get(&kpos, m));
    NB_TRY(sc.get(&nk, 1));
    k_winner_keys<<<G2, 256, 0, st>>>(P->all, flag, pos, n, C->n_rx, keys, vals);
    NB_CUDA(err, cudaGetLastError());
    NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, m,
                      bits_for((uint64_t)C->n_tx * (uint64_t)std::max(1, C->n_rx))));
    NB_CUDA(err, cudaMemsetAsync(keep, 0, m * sizeof(uint32_t), st));
    k_fresnel<<<std::min<unsigned>(grid_for(m, 64), pgrid(64)), 64, 0, st>>>(P->all, keys, vals, m, C->txd, rp.lambda,
                                                                              keep);
    NB_CUDA(err, cudaGetLastError());
    NB_TRY(exclusive_scan(sc, keep, kpos, m, nk));
    k_final<<<std::min<unsigned>(grid_for(m, 256), pgrid(256)), 256, 0, st>>>(keep, kpos, vals, m, P->final_idx);
    NB_CUDA(err, cudaGetLastError());
    uint32_t hk = 0;
    NB_CUDA(err, cudaMemcpyAsync(&hk, nk, sizeof hk, cudaMemcpyDeviceToHost, st));
    NB_CUDA(err, cudaStreamSynchronize(st));
    P->n_final = hk;
  }
  P->counts.n_paths = P->n_final;
  P->counts.n_refined_valid = -1;  // filled by a query with which = 1
  return NIMBUS_OK;
}

}  // namespace nb
