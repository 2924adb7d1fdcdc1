// Path refinement (Section 2.3): gradient descent on the path length (Eq. 2) with
// re-projection of reflection points onto the point cloud, final visibility,
// label-based and first-Fresnel-zone duplicate removal.
//
// B300 design: one warp per coarse path.  Lane k owns interaction k's state: the
// FP64 iterate (the point and, for a diffraction, its edge parameter) and its FP32
// basis; neighbours come from warp shuffles.  B300's FP64 rate is a small fraction
// of FP32, so FP64 is kept to what must accumulate without loss -- the iterate,
// the re-projected points and the path length -- while directions, gradient, local
// Hessian and step are FP32 evaluations of FP64 differences (the gradient is FP64
// again once it falls below delta, where it decides the stop).  Each re-projection
// (a ray intersected with one label's implicit surface, Eq. 1) and each final
// visibility ray uses all 32 lanes: the Eq. 1 sums are split across lanes and
// combined with shuffles, in FP32 in a frame centred on the target, and the label's
// nearby entities are cached in shared memory per interaction.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nimbus_host.hpp"
#define NB_VIS_PAIRS 0   // one load per lane and pass in the final visibility rays (see warp_geom.cuh)
#include "warp_geom.cuh"

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

__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}


// Same-label IEs near one re-projection target, cached in shared memory for each
// interaction of a warp's path.  Key: label and the target's subvoxel gR; entries
// hold the first point, the point count and a 27-bit mask of the subvoxels x around
// gR (offsets in [-1, 1]^3) whose 3x3x3 block contains the IE.  Rebuilt only when
// the key changes, i.e. when an update carries the target into another subvoxel.
// 96 entries cover a surface crossing three subvoxel layers of the 5x5x5 block (a
// noisy wall lying on subvoxel faces fills two); a fuller block makes the
// re-projection miss.
constexpr int RCAP = 96;
struct LabelCache {
  uint32_t pb[RCAP];
  uint32_t pc[RCAP];
  uint32_t nbr[RCAP];
  int gR[3];
  uint32_t label;
  int n;                 // entries, -1: empty
};

// Bit (dz+1)*9 + (dy+1)*3 + (dx+1) of the mask: an IE at subvoxel offset g from gR
// lies in the 3x3x3 block of the subvoxel at offset d iff |g - d| <= 1 per axis.
__device__ __forceinline__ uint32_t block_mask(int gx, int gy, int gz) {
  uint32_t m = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if (abs(gx - dx) <= 1 && abs(gy - dy) <= 1 && abs(gz - dz) <= 1) m |= 1u << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1);
  return m;
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// The cached entities selected for one Eq. 1 evaluation, in cache order, as a flat
// list of points: entity j holds points [beg[j], end[j]) of the list, its first one
// at pb[j] in the scene.  Per warp, in shared memory (also the scratch of fill_cache).
struct SelList {
  uint32_t end[32];
  uint32_t beg[32];
  uint32_t pb[32];
};

// (Re)build the cache for target subvoxel gR and label: the label's point IEs whose
// subvoxel lies within two subvoxels of gR -- all that Eq. 1 at any point of a
// re-projection segment around the target can draw on.  The region's voxels (z, y, x
// order; 27 for two subvoxels a voxel) are taken 32 at a time: each lane loads one
// voxel's entity range, a warp scan lays the ranges out as one flat list, and each
// lane screens two entities of every 64, so the loads of the whole region are in
// flight together instead of one voxel after another.  Entries keep the order of a
// voxel-by-voxel scan.
__device__ void fill_cache(const DScene& s, LabelCache& lc, SelList& sl, const int gR[3], uint32_t label, int lane,
                           unsigned long long& bytes) {
  int v0[3], nv[3];
  for (int a = 0; a < 3; ++a) {
    v0[a] = floor_div(gR[a] - 2, s.dv);
    nv[a] = floor_div(gR[a] + 2, s.dv) - v0[a] + 1;
  }
  const int n_vox = nv[0] * nv[1] * nv[2];
  const float ofs[3] = {s.ox, s.oy, s.oz};
  const unsigned lt = (1u << lane) - 1u;
  int nc = 0;
  for (int vb = 0; vb < n_vox; vb += 32) {
    uint32_t first = 0, cnt = 0;
    const int q = vb + lane;
    if (q < n_vox) {
      const int vx = v0[0] + q % nv[0], vy = v0[1] + (q / nv[0]) % nv[1], vz = v0[2] + q / (nv[0] * nv[1]);
      if (in_grid(s, vx, vy, vz)) {
        const uint2 cell = __ldg(&s.cells[cell_index(s, vx, vy, vz)]);
        first = cell.x;
        cnt = cell.y;
      }
    }
    uint32_t e = cnt;   // inclusive scan: the flat list's end of voxel `lane`
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, e, o);
      if (lane >= o) e += t;
    }
    const uint32_t total = __shfl_sync(FULL, e, 31);
    __syncwarp();
    sl.end[lane] = e;
    sl.beg[lane] = e - cnt;   // the voxel's start in the flat list
    sl.pb[lane] = first;      // its first entity in the scene
    __syncwarp();
    int jv0 = 0, jv1 = 0;
    for (uint32_t base = 0; base < total; base += 64) {
      bool ok[2] = {false, false};
      uint32_t pb[2] = {0, 0}, pc[2] = {0, 0}, nbr[2] = {0, 0};
      const IERec* r[2];
      float4 nm[2], rp[2];
      bool in[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint32_t t = base + 32 * u + lane;
        in[u] = t < total;
        int& jv = u == 0 ? jv0 : jv1;
        if (u == 1) jv1 = max(jv1, jv0);
        if (in[u])
          while (t >= sl.end[jv]) ++jv;
        r[u] = &s.ies[in[u] ? sl.pb[jv] + (t - sl.beg[jv]) : sl.pb[0]];
        if (in[u]) {
          nm[u] = __ldg(&r[u]->nrm_meta);
          rp[u] = __ldg(&r[u]->rp_lab);
          bytes += 32;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (in[u] && (__float_as_uint(nm[u].w) & 1u) == IE_POINT && __float_as_uint(rp[u].w) == label) {
          const float4 sc = __ldg(&r[u]->sc_pc);
          const float scv[3] = {sc.x, sc.y, sc.z};
          int dg[3];
          ok[u] = true;
          for (int a = 0; a < 3; ++a) {
            dg[a] = (int)floorf((scv[a] - ofs[a]) * s.inv_hs) - gR[a];
            ok[u] = ok[u] && abs(dg[a]) <= 2;
          }
          pc[u] = __float_as_uint(sc.w);
          nbr[u] = block_mask(dg[0], dg[1], dg[2]);
          pb[u] = __float_as_uint(__ldg(&r[u]->bbc_pb).w);
          bytes += 32;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const unsigned mask = __ballot_sync(FULL, ok[u]);
        const int slot = nc + __popc(mask & lt);
        if (ok[u] && slot < RCAP) {
          lc.pb[slot] = pb[u];
          lc.pc[slot] = pc[u];
          lc.nbr[slot] = nbr[u];
        }
        nc += __popc(mask);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    lc.gR[0] = gR[0];
    lc.gR[1] = gR[1];
    lc.gR[2] = gR[2];
    lc.label = label;
    lc.n = nc > RCAP ? RCAP + 1 : nc;
  }
  __syncwarp();
}

// Eq. 1 over the nearby points of one label -- the points of the cached IEs whose
// subvoxel lies in the 3x3x3 block around the subvoxel of x -- in FP32 in a frame
// centred on c0 (the target); xl = x - c0, dg = subvoxel of x minus gR.  The block's
// entities (at most one per subvoxel and label, so at most 27) are found with one
// ballot per 32 cache entries and laid out as one flat list of their points; lane l
// takes points l and l + 32 of every 64 of it, so every lane has two points' loads
// in flight and no lane idles at an entity's end.  Every lane returns the same f
// and normal.  REFINE_PTS is the number of points (loads in flight) per lane and pass.
#ifndef REFINE_PTS
#define REFINE_PTS 2
#endif
__device__ bool sdf_label_warp(const DScene& s, const LabelCache& lc, SelList& sl, float3 xl, const int dg[3],
                               float3 c0, float* f, float3* n_out, int lane, unsigned long long& bytes) {
  if (abs(dg[0]) > 1 || abs(dg[1]) > 1 || abs(dg[2]) > 1) return false;
  const int di = (dg[2] + 1) * 9 + (dg[1] + 1) * 3 + dg[0] + 1;
  const int nc = lc.n;
  static_assert(RCAP <= 96, "three ballots cover the cache");
  const bool b0 = lane < nc && ((lc.nbr[lane] >> di) & 1u);
  const bool b1 = 32 + lane < nc && ((lc.nbr[32 + lane] >> di) & 1u);
  const bool b2 = 64 + lane < nc && ((lc.nbr[64 + lane] >> di) & 1u);
  const unsigned sel0 = __ballot_sync(FULL, b0), sel1 = __ballot_sync(FULL, b1), sel2 = __ballot_sync(FULL, b2);
  const unsigned lt = (1u << lane) - 1u;
  const int n0 = __popc(sel0), n01 = n0 + __popc(sel1), ns = n01 + __popc(sel2);
  // entity j of the list: its first point and count, written by the lane that holds it
  if (b0) { sl.pb[__popc(sel0 & lt)] = lc.pb[lane]; sl.beg[__popc(sel0 & lt)] = lc.pc[lane]; }
  if (b1) { sl.pb[n0 + __popc(sel1 & lt)] = lc.pb[32 + lane]; sl.beg[n0 + __popc(sel1 & lt)] = lc.pc[32 + lane]; }
  if (b2) { sl.pb[n01 + __popc(sel2 & lt)] = lc.pb[64 + lane]; sl.beg[n01 + __popc(sel2 & lt)] = lc.pc[64 + lane]; }
  __syncwarp();
  const uint32_t pc = lane < ns ? sl.beg[lane] : 0u;
  uint32_t e = pc;   // inclusive scan of the counts: the list end of entity `lane`
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, e, o);
    if (lane >= o) e += t;
  }
  const uint32_t total = __shfl_sync(FULL, e, 31);
  __syncwarp();
  sl.end[lane] = e;
  sl.beg[lane] = e - pc;
  __syncwarp();
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int j[REFINE_PTS];
#pragma unroll
  for (int u = 0; u < REFINE_PTS; ++u) j[u] = 0;
  for (uint32_t base = 0; base < total; base += 32 * REFINE_PTS) {
    float4 P[REFINE_PTS], N[REFINE_PTS];
    bool in[REFINE_PTS];
#pragma unroll
    for (int u = 0; u < REFINE_PTS; ++u) {
      const uint32_t q = base + 32 * u + lane;
      in[u] = q < total;
      if (u > 0) j[u] = max(j[u], j[u - 1]);
      if (in[u])
        while (q >= sl.end[j[u]]) ++j[u];
      // past the list's end: re-read a point of the list, unused
      const uint32_t a = in[u] ? sl.pb[j[u]] + (q - sl.beg[j[u]]) : sl.pb[0];
      P[u] = __ldg(&s.pts[a]);
      N[u] = __ldg(&s.pnrm[a]);
    }
#pragma unroll
    for (int u = 0; u < REFINE_PTS; ++u)
      if (in[u]) eq1_term(v, xl, P[u], N[u], c0, s.sdf_inv_s2);
  }
  __syncwarp();
  if (lane == 0) bytes += 24ull * total;
  wsum8(v, lane);
  return eq1_finish(v, xl, f, n_out);
}

// Subvoxel of c0 + xl relative to gR.
// Continuous points of the refinement are binned in FP32 with the reciprocal of h_s;
// the target's own subvoxel gR uses the same expression, so dg = 0 at the target.
__device__ __forceinline__ void rel_subvoxel(const DScene& s, float3 c0, float3 xl, const int gR[3], int dg[3]) {
  dg[0] = (int)floorf((c0.x - s.ox + xl.x) * s.inv_hs) - gR[0];
  dg[1] = (int)floorf((c0.y - s.oy + xl.y) * s.inv_hs) - gR[1];
  dg[2] = (int)floorf((c0.z - s.oz + xl.z) * s.inv_hs) - gR[2];
}

// Re-projection (Section 2.3): the ray from P toward the updated point R is
// intersected with the implicit surface of label `label` (Eq. 1 over nearby points of
// that label) on a segment of one subvoxel diameter centred on R.  Eq. 1 is evaluated
// at R first: where R already lies on the surface (|f| < eps, as it does once a path
// nears its stationary point) the hit is one Newton step along the ray from R, if that
// stays on the segment, with Eq. 1's normal at R; otherwise the segment is marched
// from its near end (Section 2.2.1) and the normal is evaluated at the hit.  The
// evaluations run in FP32 relative to R; the new point is R plus the FP32 offset along
// the ray, in FP64.
__device__ bool reproject_warp(const DScene& s, const d3* Pp, const d3* Rp, uint32_t label, d3* c_out, float3* n_out,
                               int lane, unsigned long long& bytes, LabelCache& lc, SelList& sl) {
  const d3 P = *Pp, R = *Rp;
  const float3 dvf = tof(R - P);
  const float tR = len(dvf);                // FP32: only compared with offsets of the segment
  if (!(tR > 1e-9f)) return false;
  const float3 d = (1.f / tR) * dvf;
  const float3 c0 = tof(R);
  const float3 r0 = tof(R - tod(c0));      // R relative to its FP32 rounding
  const int zero[3] = {0, 0, 0};
  int gR[3];
  rel_subvoxel(s, c0, r0, zero, gR);
  if (lc.n < 0 || lc.label != label || lc.gR[0] != gR[0] || lc.gR[1] != gR[1] || lc.gR[2] != gR[2])
    fill_cache(s, lc, sl, gR, label, lane, bytes);
  if (lc.n > RCAP || lc.n == 0) return false;
  const float half = 0.5f * s.seg_len;
  float th = 0.f, f;
  float3 n;
  int dg[3];
  auto eval = [&](float t, float* fo, float3* no) {
    float3 x = r0 + t * d;
    int g[3];
    rel_subvoxel(s, c0, x, gR, g);
    return sdf_label_warp(s, lc, sl, x, g, c0, fo, no, lane, bytes);
  };
  {
    float fR;
    float3 nR;
    if (eval(0.f, &fR, &nR) && fabsf(fR) < s.sdf_eps) {
      const float dn = dot(nR, d);
      const float t1 = fabsf(dn) > 1e-3f ? -fR / dn : 0.f;
      if (tR + t1 > 0.f && fabsf(t1) <= half) {
        *c_out = *Rp + (double)t1 * tod(d);
        *n_out = nR;
        return true;
      }
    }
  }
  if (!march_abs_f<false>(eval, d, -half, half, s.sdf_eps, s.sdf_max_steps, &th)) return false;
  // the placed hit must stay on the marched segment (and in front of P)
  if (!(tR + th > 0.f) || fabsf(th) > half) return false;
  float3 xl = r0 + th * d;
  rel_subvoxel(s, c0, xl, gR, dg);
  if (!sdf_label_warp(s, lc, sl, xl, dg, c0, &f, &n, lane, bytes)) return false;
  *c_out = *Rp + (double)th * tod(d);
  *n_out = n;
  return true;
}

// One warp per coarse path: lanes 1..n hold the interactions, lane 0 the TX and
// lane n+1 the RX.  Iterate rho times (or until ||grad f|| < grad_stop): gradient of
// Eq. 2 per interaction, a Jacobi step (each interaction's gradient scaled by its
// local inverse Hessian times gamma) clamped to h_s, then for each reflection a
// re-projection ray from the previous interaction point toward
// R_k = c_k + r_k u_k + s_k v_k, for each diffraction D_k = c_k + t_k w_k.
// Precision: the iterate (interaction points, edge parameters), the re-projected
// points and the path length are FP64; directions, gradient, local Hessian and step
// are FP32 evaluations from FP64 differences, except that once ||grad|| < delta the
// gradient that decides the stop and drives the last steps is FP64.
// Occupancy: six 4-warp blocks per SM (80 registers a thread; 8.3 KB of static and
// 14 KB of dynamic shared memory a block for three reflections).  The kernel is bound
// by latency: resident warps pay most (measured with the flat point list on the
// indoor and noisy-room workloads: 2 points per lane and 6 blocks 5.08 / 2.71 s, 3
// and 6 4.80 / 2.79 s, 4 and 5 5.14 / 2.96 s, 3 and 5 5.31 / 2.93 s), and any
// sizeable register spill in the point loop costs more than any of it.  So each
// path's FP64 state lives in shared memory (WarpPath), indexed by node (0 = TX,
// n+1 = RX), and is read where it is used.
struct WarpPath {
  d3 I[NB_MAXI + 2], c[NB_MAXI + 2], R[NB_MAXI + 2], In[NB_MAXI + 2], p0[NB_MAXI + 2];
  double tpar[NB_MAXI + 2];
  float3 u[NB_MAXI + 2], v[NB_MAXI + 2], w[NB_MAXI + 2];
  float elen[NB_MAXI + 2];
};

// Two-phase refinement (a launch layout; results are the same bit for bit).  Phase 1
// runs every path for at most `cap` iterations; a path still running then saves its
// iterate and leaves.  Phase 2 resumes those paths, longest first by one of two
// rankings: the cost per iteration so far, or the predicted remaining time (that cost
// times the iterations still needed at the gradient's rate of decrease over the second
// half of phase 1), so the long ones start at the beginning of a launch instead of
// wherever the hand-out order put them.  A resumed path continues the same iteration sequence from
// the same FP64 state; its label caches are refilled, and a cache's content is a
// function of its key only.
struct PathState {
  d3 I[NB_MAXI + 2];      // iterate (nodes 0..n+1)
  d3 c[NB_MAXI + 2];      // re-projected points / edge base points
  double tpar[NB_MAXI + 2];
  float3 u[NB_MAXI + 2], v[NB_MAXI + 2];
  int it;
};

struct RefineSplit {
  int phase;              // 0: one pass; 1: stop at cap; 2: resume the saved paths
  int cap;
  int key;                // resume order: 0 cost per iteration, 1 predicted remaining time
  PathState* st;          // [n] by coarse index
  uint32_t* cont;         // phase 1: coarse indices of the saved paths; phase 2: in resume order
  uint64_t* cont_key;     // phase 1: 2^40 - 1 minus the predicted remaining time (ascending sort = longest first)
  unsigned* cont_n;
};

#ifndef REFINE_BLOCKS_PER_SM
#define REFINE_BLOCKS_PER_SM 6
#endif
__global__ void __launch_bounds__(128, REFINE_BLOCKS_PER_SM) k_refine(DScene s, DRefine rp, CoarseView C, const double* txd,
                                                   const double* rxd, ExactRec* out, unsigned long long* bytes_out,
                                                   unsigned long long* next_path, const uint32_t* order, int n_cache,
                                                   RefineSplit sp) {
  // label caches: n_cache per warp (the trace's reflection limit), in dynamic shared
  // memory, so that the rest of the SM's 256 KB stays L1 for the point loads
  extern __shared__ LabelCache s_dyn[];
  __shared__ WarpPath s_path[4];
  __shared__ SelList s_sel[4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  LabelCache* cache = s_dyn + wib * n_cache;
  WarpPath& W = s_path[wib];
  unsigned long long bytes = 0;
  for (;;) {
    unsigned long long grab = 0;
    if (lane == 0) grab = atomicAdd(next_path, 1ull);
    const int64_t gi = (int64_t)__shfl_sync(FULL, grab, 0);
    const int64_t n_work = sp.phase == 2 ? (int64_t)*(volatile unsigned*)sp.cont_n : C.n;
    if (gi >= n_work) break;
    const int64_t i = sp.phase == 2 ? (int64_t)sp.cont[gi] : (order ? order[gi] : gi);
    const int n = (int)C.nint[i];
    const uint32_t types = C.types[i];
    const uint32_t tx = C.tx[i], rx = C.rx[i];
    const bool mine = lane >= 1 && lane <= n;
    const bool node = lane <= n + 1;
    const bool diff = mine && ((types >> (lane - 1)) & 1u);
    if (lane < n_cache) cache[lane].n = -1;
    uint32_t my_lab = NB_NONE_LABEL, my_ie = 0xffffffffu;
    uint8_t my_mat = 255;
    if (lane == 0) W.I[0] = D3(txd[3 * tx], txd[3 * tx + 1], txd[3 * tx + 2]);
    if (lane == n + 1) W.I[n + 1] = D3(rxd[3 * rx], rxd[3 * rx + 1], rxd[3 * rx + 2]);
    if (mine) {
      my_ie = C.ie[i * NB_MAXI + lane - 1];
      my_lab = C.lab[i * NB_MAXI + lane - 1];
      const IERec* r = &s.ies[my_ie];
      float4 rpl = r->rp_lab, nm = r->nrm_meta;
      my_mat = (uint8_t)((__float_as_uint(nm.w) >> 8) & 0xffu);
      W.c[lane] = D3(rpl.x, rpl.y, rpl.z);
      W.I[lane] = W.c[lane];
      W.tpar[lane] = 0.0;
      if (!diff) {
        float3 u, v;
        onb(normalize(xyz(nm)), &u, &v);
        W.u[lane] = u;
        W.v[lane] = v;
      } else {
        const double* E = s.edges + 12 * __float_as_uint(r->bbc_pb.w);
        W.p0[lane] = D3(E[0], E[1], E[2]);
        d3 ev = D3(E[3] - E[0], E[4] - E[1], E[5] - E[2]);
        double el = len(ev);
        W.elen[lane] = (float)el;
        W.w[lane] = tof((1.0 / el) * ev);
      }
    }
    __syncwarp();
    int status = ST_VALID, it = 0;
    bool converged = false;
    if (sp.phase == 2) {
      const PathState& ps = sp.st[i];
      if (node) W.I[lane] = ps.I[lane];
      if (mine) {
        W.c[lane] = ps.c[lane];
        W.tpar[lane] = ps.tpar[lane];
        W.u[lane] = ps.u[lane];
        W.v[lane] = ps.v[lane];
      }
      it = ps.it;
      __syncwarp();
    }
    const long long t_path = clock64();
    bool saved = false;
    float g_half = 0.f;   // phase 1: the gradient norm half-way to the cap
    float gn = 0.f;
    for (; it <= rp.rho; ++it) {
      if (sp.phase == 1 && it == sp.cap) {
        // phase 1 ends here for this path: save the iterate for phase 2
        PathState& ps = sp.st[i];
        if (node) ps.I[lane] = W.I[lane];
        if (mine) {
          ps.c[lane] = W.c[lane];
          ps.tpar[lane] = W.tpar[lane];
          ps.u[lane] = W.u[lane];
          ps.v[lane] = W.v[lane];
        }
        if (lane == 0) {
          ps.it = it;
          const unsigned slot = atomicAdd(sp.cont_n, 1u);
          // predicted remaining time: cost per iteration so far times the iterations
          // still needed at the gradient's rate of decrease over the second half of
          // phase 1 (rho - it when it did not decrease)
          const double per_it = (double)(clock64() - t_path) / (double)max(1, sp.cap);
          double rem = sp.key == 0 ? 1.0 : (double)(rp.rho - it);
          if (sp.key == 1 && g_half > 0.f && gn > 0.f && gn < g_half) {
            const double rate = log((double)gn / (double)g_half) / (double)max(1, it - sp.cap / 2);
            rem = fmin(rem, fmax(1.0, log(rp.grad_stop / (double)gn) / rate));
          }
          const double cost = fmin(per_it * rem / 64.0, (double)((1ull << 40) - 1));
          sp.cont[slot] = (uint32_t)i;
          sp.cont_key[slot] = (1ull << 40) - 1 - (uint64_t)cost;
        }
        saved = true;
        break;
      }
      // gradient of Eq. 2: (e_in + e_out) . (u, v) for reflections, . w for diffractions
      float g0 = 0.f, g1 = 0.f, a = 1.f, b = 1.f;
      float3 ea = f3(0, 0, 0), eb = f3(0, 0, 0);
      if (mine) {
        const d3 I = W.I[lane];
        float3 fa = tof(I - W.I[lane - 1]), fb = tof(I - W.I[lane + 1]);
        a = len(fa);
        b = len(fb);
        ea = a > 0.f ? (1.f / a) * fa : fa;
        eb = b > 0.f ? (1.f / b) * fb : fb;
        float3 e = ea + eb;
        if (!diff) {
          g0 = dot(e, W.u[lane]);
          g1 = dot(e, W.v[lane]);
        } else {
          g0 = dot(e, W.w[lane]);
        }
      }
      gn = sqrtf(wsum(g0 * g0 + g1 * g1));
      // Near the stop the gradient is taken again in FP64: at grazing incidence the
      // local length is nearly flat along the surface, so an FP32 gradient (error
      // ~1e-7) would move the stopping point by millimetres along it.
      if (gn < (float)rp.delta) {
        double h0 = 0.0, h1 = 0.0;
        if (mine) {
          const d3 I = W.I[lane];
          const d3 fa = I - W.I[lane - 1], fb = I - W.I[lane + 1];
          const d3 e = (1.0 / len(fa)) * fa + (1.0 / len(fb)) * fb;
          if (!diff) {
            h0 = dot(e, tod(W.u[lane]));
            h1 = dot(e, tod(W.v[lane]));
          } else {
            h0 = dot(e, tod(W.w[lane]));
          }
        }
        g0 = (float)h0;
        g1 = (float)h1;
        gn = (float)sqrt(wsumd(h0 * h0 + h1 * h1));
      }
      if (gn < (float)rp.grad_stop) {
        converged = true;
        break;
      }
      if (sp.phase == 1 && it == sp.cap / 2) g_half = gn;
      if (it == rp.rho) break;
      bool off = false;
      if (node) W.In[lane] = W.I[lane];
      // step: gradient scaled by the inverse Hessian of the local length f_k (2x2 in
      // (r, s), 1x1 in t) times gamma; near-singular Hessians fall back to eta
      const float hsum = 1.f / a + 1.f / b;
      const float gam = (float)rp.gamma, eta = gam / hsum, hs = (float)rp.hs;
      if (mine && !diff) {
        const float3 u = W.u[lane], v = W.v[lane];
        float au = dot(ea, u), av = dot(ea, v), bu = dot(eb, u), bv = dot(eb, v);
        float h11 = (1.f - au * au) / a + (1.f - bu * bu) / b;
        float h22 = (1.f - av * av) / a + (1.f - bv * bv) / b;
        float h12 = -(au * av) / a - (bu * bv) / b;
        float det = h11 * h22 - h12 * h12;
        float rr, ss;
        if (det > 1e-12f * hsum * hsum) {
          rr = -gam * (h22 * g0 - h12 * g1) / det;
          ss = -gam * (h11 * g1 - h12 * g0) / det;
        } else {
          rr = -eta * g0;
          ss = -eta * g1;
        }
        float l = sqrtf(rr * rr + ss * ss);
        if (l > hs) {
          rr *= hs / l;
          ss *= hs / l;
        }
        W.R[lane] = W.c[lane] + (double)rr * tod(u) + (double)ss * tod(v);   // R_k = c_k + r_k u_k + s_k v_k
      }
      if (diff) {
        const float3 w = W.w[lane];
        float aw = dot(ea, w), bw = dot(eb, w);
        float hw = (1.f - aw * aw) / a + (1.f - bw * bw) / b;
        float dt = hw > 1e-12f * hsum ? -gam * g0 / hw : -eta * g0;
        if (fabsf(dt) > hs) dt = copysignf(hs, dt);
        const double tp = W.tpar[lane] + (double)dt;            // D_k = c_k + t_k w_k
        W.tpar[lane] = tp;
        const d3 Dn = W.c[lane] + tp * tod(w);
        W.In[lane] = Dn;
        double along = dot(Dn - W.p0[lane], tod(w));
        off = along < 0.0 || along > (double)W.elen[lane];
      }
      if (__any_sync(FULL, off)) {
        status = ST_OFF_EDGE;
        break;
      }
      __syncwarp();
      for (int k = 1; k <= n; ++k) {
        if ((types >> (k - 1)) & 1u) continue;
        uint32_t lk = __shfl_sync(FULL, my_lab, k);
        d3 cn;
        float3 nn;
        // the cache of the path's r-th reflection, r = reflections before interaction k
        const int r = (k - 1) - __popc(types & ((1u << (k - 1)) - 1u));
        if (r >= n_cache) {   // more reflections than the trace allowed: not a path of this trace
          status = ST_MISS;
          break;
        }
        if (!reproject_warp(s, &W.I[k - 1], &W.R[k], lk, &cn, &nn, lane, bytes, cache[r], s_sel[wib])) {
          status = ST_MISS;
          break;
        }
        if (lane == k) {
          W.c[k] = cn;
          float3 u, v;
          onb(normalize(nn), &u, &v);
          W.u[k] = u;
          W.v[k] = v;
          W.In[k] = cn;
        }
      }
      if (status != ST_VALID) break;
      __syncwarp();
      if (node) W.I[lane] = W.In[lane];
      __syncwarp();
    }
    __syncwarp();
    if (saved) continue;
    if (status == ST_VALID && !converged && !(gn < (float)rp.delta)) status = ST_NOT_CONVERGED;
    if (status == ST_VALID) {
      // visibility between consecutive path nodes
      for (int k = 0; k <= n; ++k) {
        float3 A = tof(W.I[k]), B = tof(W.I[k + 1]);
        uint32_t la = __shfl_sync(FULL, my_lab, k), lb = __shfl_sync(FULL, my_lab, min(k + 1, 31));
        Endpoint ea{IGN_NONE, NB_NONE_LABEL}, eb{IGN_NONE, NB_NONE_LABEL};
        if (k >= 1) ea = Endpoint{((types >> (k - 1)) & 1u) ? IGN_ANY : IGN_LABEL, la};
        if (k + 1 <= n) eb = Endpoint{((types >> k) & 1u) ? IGN_ANY : IGN_LABEL, lb};
        if (!visible_warp(s, A, B, ea, eb, lane, bytes)) {
          status = ST_OCCLUDED;
          break;
        }
      }
    }
    double seg = lane <= n ? len(W.I[lane + 1] - W.I[lane]) : 0.0;
    double L = wsumd(seg);
    ExactRec* o = &out[i];
    if (lane == 0) {
      o->length = status == ST_VALID ? L : 0.0;
      o->delay = o->length / C_LIGHT;
      o->grad = (double)gn;
      o->tx = tx;
      o->rx = rx;
      o->n = (uint32_t)n;
      o->types = types;
      o->status = (uint32_t)status;
      o->iters = (uint32_t)it;
      o->gid = C.gid[i];
      o->pad = 0;
    }
    if (lane >= 1 && lane <= NB_MAXI) {
      int q = lane - 1;
      const d3 I = mine ? W.I[lane] : D3(0, 0, 0);
      o->lab[q] = mine ? my_lab : NB_NONE_LABEL;
      o->ie[q] = mine ? my_ie : 0xffffffffu;
      o->mat[q] = mine ? my_mat : 255;
      o->pts[q][0] = I.x;
      o->pts[q][1] = I.y;
      o->pts[q][2] = I.z;
    }
    __syncwarp();
  }
  // each lane counted its own share of the records read
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(FULL, bytes, o);
  if (lane == 0 && bytes) atomicAdd(bytes_out, bytes);
}

// Hand-out order of the paths (it changes no result, only which paths run last).
// Mode 1: the paths with the most interactions first.  Mode 2: first the paths whose
// re-projection rays graze their surfaces at the starting iterate (the smallest
// |n . d| over the reflections, in 16 buckets of 0.05), then by interactions.  A
// re-projection ray nearly tangent to its surface marches in small |f| steps, and the
// paths that keep such a ray while they run all rho iterations take hundreds of
// milliseconds each; started last, they decide when the launch ends.  On the noisy
// room the paths starting below 0.2 are a fifth of the paths and hold a third of the
// oracle's Eq. 1 evaluations and most of the heaviest paths.
__global__ void k_order_keys(DScene s, CoarseView C, const double* txd, const double* rxd, int mode, uint64_t* keys,
                             uint32_t* vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t n = C.nint[i];
    uint64_t key = (uint64_t)(NB_MAXI - n);
    if (mode == 2) {
      const uint32_t t = C.tx[i];
      float3 prev = f3((float)txd[3 * t], (float)txd[3 * t + 1], (float)txd[3 * t + 2]);
      float gmin = 1.f;
      for (uint32_t q = 0; q < n && q < NB_MAXI; ++q) {
        const IERec* r = &s.ies[C.ie[i * NB_MAXI + q]];
        const float3 rp = xyz(__ldg(&r->rp_lab));
        if (!((C.types[i] >> q) & 1u)) {
          const float3 d = rp - prev;
          const float dl = len(d);
          if (dl > 0.f) gmin = fminf(gmin, fabsf(dot(d, xyz(__ldg(&r->nrm_meta)))) / dl);
        }
        prev = rp;
      }
      key += (uint64_t)min(15, (int)(gmin * 20.f)) << 4;
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
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

// Is B inside the first Fresnel zones of the kept path A (same chain of interaction
// types, every interaction point of B within the zone radius around A's)?
__device__ bool in_fresnel_zones(const ExactRec& A, const ExactRec& B, const double* txd, double lambda) {
  if (A.n != B.n || A.n == 0 || A.types != B.types) return false;
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
  return inside;
}

// One warp per TX/RX pair (the pair whose first entry lies in the warp's chunk of 32
// positions): order its label winners by path_less into svals -- a total order there,
// since the winners of one pair differ in their type or label sequence, so each
// winner's rank is the number of winners before it -- then, in that order, drop every
// path whose interaction points all lie in the first Fresnel zones of an earlier kept
// path with the same chain of interaction types, the lanes testing the earlier kept
// paths together.  The order and every decision are those of one thread sorting the
// pair and then passing over it.
__global__ void k_fresnel(const ExactRec* ex, const uint64_t* keys, const uint32_t* vals, int64_t n,
                          const double* txd, double lambda, uint32_t* svals, uint32_t* keep) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < n; base += n_warps * 32) {
    const int64_t my = base + lane;
    const bool start = my < n && (my == 0 || keys[my] != keys[my - 1]);
    unsigned sm = __ballot_sync(FULL, start);
    while (sm) {
      const int64_t i = base + __ffs(sm) - 1;
      sm &= sm - 1;
      int64_t e = i + 1;   // end of the pair: the first later entry with another key
      for (;;) {
        const int64_t q = e + lane;
        const unsigned om = __ballot_sync(FULL, q >= n || keys[q] != keys[i]);
        if (om) {
          e += __ffs(om) - 1;
          break;
        }
        e += 32;
      }
      for (int64_t a = i + lane; a < e; a += 32) {
        const ExactRec& X = ex[vals[a]];
        int64_t r = 0;
        for (int64_t b = i; b < e; ++b) {   // ties (none are expected) by position: a permutation
          const ExactRec& Y = ex[vals[b]];
          if (b != a && (path_less(Y, X) || (b < a && !path_less(X, Y)))) ++r;
        }
        svals[i + r] = vals[a];
      }
      __syncwarp();
      for (int64_t bI = i; bI < e; ++bI) {
        const ExactRec& B = ex[svals[bI]];
        bool dup = false;
        for (int64_t aI = i + lane; aI < bI && !dup; aI += 32)
          dup = keep[aI] && in_fresnel_zones(ex[svals[aI]], B, txd, lambda);
        dup = __any_sync(FULL, dup);
        if (lane == 0) keep[bI] = dup ? 0u : 1u;
        __syncwarp();
      }
    }
  }
}

// Entries of the continuation list past its count sort after every saved path.
__global__ void k_cont_fill(uint64_t* keys, uint32_t* vals, const unsigned* cnt, int64_t n) {
  const int64_t m = *cnt;
  for (int64_t i = m + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = 1ull << 40;
    vals[i] = 0u;
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

int refine_paths(Mem& mem, SceneObj* S, CoarseObj* C, const nimbus_refine_params* p, PathsObj* P, cudaStream_t st,
                 const Tuning& tn) {
  std::string* err = mem.err;
  if (!(p->delta > 0) || p->rho < 0 || !(p->gamma > 0) || !(p->freq_hz > 0)) {
    *err = "refine: invalid parameters";
    return NIMBUS_ERR_ARG;
  }
  const long long launches0 = g_launches.load();
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
  Scratch sc(&mem, st);
  unsigned long long* rbytes;   // [0] bytes read, [1] next path to hand out
  NB_TRY(sc.get(&rbytes, 2));
  // two-phase layout: state, continuation list and its sort buffers
  const bool split = tn.refine_split > 0 && tn.refine_split < p->rho;
  RefineSplit sp1{}, sp2{}, sp0{};
  uint64_t* ck_alt = nullptr;
  uint32_t* cv_alt = nullptr;
  if (split) {
    PathState* st_buf;
    uint32_t* cont;
    uint64_t* ckey;
    unsigned* cnt;
    NB_TRY(sc.get(&st_buf, n));
    NB_TRY(sc.get(&cont, n));
    NB_TRY(sc.get(&ckey, n));
    NB_TRY(sc.get(&cnt, 1));
    NB_TRY(sc.get(&ck_alt, n));
    NB_TRY(sc.get(&cv_alt, n));
    sp1 = RefineSplit{1, tn.refine_split, tn.refine_split_key, st_buf, cont, ckey, cnt};
    sp2 = RefineSplit{2, tn.refine_split, tn.refine_split_key, st_buf, cont, ckey, cnt};
  }
  const int n_cache = std::max(1, std::min(C->max_refl, NB_MAXI));
  const size_t dyn = sizeof(LabelCache) * 4 * n_cache;
  int refine_blocks = 0;   // resident blocks per SM (a persistent grid)
  NB_CUDA(err, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&refine_blocks, k_refine, 128, dyn));
  if (tn.refine_blocks > 0) refine_blocks = std::min(refine_blocks, tn.refine_blocks);
  const unsigned G = std::min<unsigned>(grid_for(n * 32, 128), (unsigned)(num_sms() * std::max(1, refine_blocks)));
  // hand out the paths with the most interactions first (they run longest), so the
  // launch does not end on a few long paths
  uint64_t *okeys = nullptr, *okeys_alt = nullptr;
  uint32_t *ovals = nullptr, *ovals_alt = nullptr;
  if (tn.refine_order) {
    NB_TRY(sc.get(&okeys, n));
    NB_TRY(sc.get(&okeys_alt, n));
    NB_TRY(sc.get(&ovals, n));
    NB_TRY(sc.get(&ovals_alt, n));
  }
  unsigned long long* best;
  uint32_t *widx, *flag, *pos, *nw;
  const uint32_t ng = C->n_groups_cap;
  NB_TRY(sc.get(&best, ng));
  NB_TRY(sc.get(&widx, ng));
  NB_TRY(sc.get(&flag, n));
  NB_TRY(sc.get(&pos, n));
  NB_TRY(sc.get(&nw, 1));
  const size_t arena_bytes = (tn.refine_order ? radix_arena_bytes(n, 8) : 0) + scan_arena_bytes(n, true) +
                             (split ? radix_arena_bytes(n, 41) : 0);
  char* arena;
  NB_TRY(sc.get(&arena, std::max<size_t>(1, arena_bytes)));
  const unsigned G2 = std::min<unsigned>(grid_for(n, 256), pgrid(256));
  StageTimer tm(st);
  const int e0 = stretch_event(tm, mem, GRAPH_REFINE, 0), e1 = stretch_event(tm, mem, GRAPH_REFINE, 1),
            e3 = stretch_event(tm, mem, GRAPH_DEDUP, 0);
  // refinement, final visibility and the per-group winners: one stretch with no host
  // round trip (one CUDA graph by default)
  NB_TRY(run_stretch(mem, st, tn.graph != 0, GRAPH_REFINE, [&](cudaStream_t q) -> int {
    Scratch ws(&mem, q);
    ws.arena = arena;
    ws.arena_cap = arena_bytes;
    NB_CUDA(err, cudaMemsetAsync(rbytes, 0, 2 * sizeof(unsigned long long), q));
    tm.record(e0, q);
    if (tn.refine_order) {
      k_order_keys<<<grid_for(n, 256), 256, 0, q>>>(S->d, cv, C->txd, C->rxd, tn.refine_order, okeys, ovals);
      NB_LAUNCHED(err);
      NB_TRY(radix_sort(ws, okeys, ovals, okeys_alt, ovals_alt, n, 8));
    }
    if (!split) {
      k_refine<<<G, 128, dyn, q>>>(S->d, rp, cv, C->txd, C->rxd, P->all, rbytes, rbytes + 1, ovals, n_cache, sp0);
      NB_LAUNCHED(err);
    } else {
      NB_CUDA(err, cudaMemsetAsync(sp1.cont_n, 0, sizeof(unsigned), q));
      k_refine<<<G, 128, dyn, q>>>(S->d, rp, cv, C->txd, C->rxd, P->all, rbytes, rbytes + 1, ovals, n_cache, sp1);
      NB_LAUNCHED(err);
      k_cont_fill<<<grid_for(n, 256), 256, 0, q>>>(sp1.cont_key, sp1.cont, sp1.cont_n, n);
      NB_LAUNCHED(err);
      NB_TRY(radix_sort(ws, sp1.cont_key, sp1.cont, ck_alt, cv_alt, n, 41));
      NB_CUDA(err, cudaMemsetAsync(rbytes + 1, 0, sizeof(unsigned long long), q));
      k_refine<<<G, 128, dyn, q>>>(S->d, rp, cv, C->txd, C->rxd, P->all, rbytes, rbytes + 1, ovals, n_cache, sp2);
      NB_LAUNCHED(err);
    }
    tm.record(e1, q);
    NB_CUDA(err, cudaMemsetAsync(best, 0xff, ng * sizeof(unsigned long long), q));
    NB_CUDA(err, cudaMemsetAsync(widx, 0xff, ng * sizeof(uint32_t), q));
    k_best_len<<<G2, 256, 0, q>>>(P->all, n, best);
    NB_LAUNCHED(err);
    k_best_idx<<<G2, 256, 0, q>>>(P->all, n, best, widx);
    NB_LAUNCHED(err);
    k_winner_flags<<<G2, 256, 0, q>>>(P->all, n, widx, flag);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(ws, flag, pos, n, nw));
    return NIMBUS_OK;
  }));
  // valid paths count (for the counters)
  uint32_t hw = 0;
  unsigned long long hb = 0;
  NB_CUDA(err, cudaMemcpyAsync(&hw, nw, sizeof hw, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaMemcpyAsync(&hb, rbytes, sizeof hb, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t m = hw;
  bool deduped = false;
  if (m > 0) {
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt, *svals, *keep, *kpos, *nk;
    NB_TRY(sc.get(&keys, m));
    NB_TRY(sc.get(&keys_alt, m));
    NB_TRY(sc.get(&vals, m));
    NB_TRY(sc.get(&vals_alt, m));
    NB_TRY(sc.get(&svals, m));
    NB_TRY(sc.get(&keep, m));
    NB_TRY(sc.get(&kpos, m));
    NB_TRY(sc.get(&nk, 1));
    const int key_bits = bits_for((uint64_t)C->n_tx * (uint64_t)std::max(1, C->n_rx));
    const size_t arena2 = radix_arena_bytes(m, key_bits) + scan_arena_bytes(m, true);
    char* arena_d;
    NB_TRY(sc.get(&arena_d, std::max<size_t>(1, arena2)));
    // label and first-Fresnel-zone dedup of the winners: a second stretch
    NB_TRY(run_stretch(mem, st, tn.graph != 0, GRAPH_DEDUP, [&](cudaStream_t q) -> int {
      Scratch ws(&mem, q);
      ws.arena = arena_d;
      ws.arena_cap = arena2;
      k_winner_keys<<<G2, 256, 0, q>>>(P->all, flag, pos, n, C->n_rx, keys, vals);
      NB_LAUNCHED(err);
      NB_TRY(radix_sort(ws, keys, vals, keys_alt, vals_alt, m, key_bits));
      NB_CUDA(err, cudaMemsetAsync(keep, 0, m * sizeof(uint32_t), q));
      k_fresnel<<<std::min<unsigned>(grid_for((m + 31) / 32 * 32, 256), pgrid(256)), 256, 0, q>>>(
          P->all, keys, vals, m, C->txd, rp.lambda, svals, keep);
      NB_LAUNCHED(err);
      NB_TRY(exclusive_scan(ws, keep, kpos, m, nk));
      k_final<<<std::min<unsigned>(grid_for(m, 256), pgrid(256)), 256, 0, q>>>(keep, kpos, svals, m, P->final_idx);
      NB_LAUNCHED(err);
      tm.record(e3, q);
      return NIMBUS_OK;
    }));
    deduped = true;
    uint32_t hk = 0;
    NB_CUDA(err, cudaMemcpyAsync(&hk, nk, sizeof hk, cudaMemcpyDeviceToHost, st));
    NB_CUDA(err, cudaStreamSynchronize(st));
    P->n_final = hk;
  }
  P->counts.n_paths = P->n_final;
  P->counts.n_refined_valid = -1;  // filled by a query with which = 1
  P->counts.ms_refine = tm.ms(e0, e1);
  P->counts.ms_dedup = deduped ? tm.ms(e1, e3) : 0.0;
  P->counts.bytes_refine = (int64_t)hb;
  P->counts.launches = C->counts.launches + (g_launches.load() - launches0);
  return NIMBUS_OK;
}

}  // namespace nb
