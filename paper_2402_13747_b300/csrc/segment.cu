// Automatic surface labels and exterior edges for unlabelled clouds.
//
// The paper's method starts from a labelled cloud: its labels come from a
// segmentation whose clusters are distinct surfaces (Section 2; Section 3 used a
// plane-fitting algorithm from PCL) and its diffraction edges are inserted by hand
// (Section 2).  This file runs the reading of both steps that nimbus.h states with
// nimbus_segment, on the voxelisation of the cloud under a single label, so that each
// IE is the point group of one subvoxel (Section 2.1) in (voxel, subvoxel) order and
// its points keep their input order.
//
// Work per group is a thread: a few tens of points, FP64 moments in point order, a
// 3x3 Jacobi eigen-solve.  Surfaces are the connected components of the join graph,
// found by a lock-free union-find that always hooks the larger root under the smaller,
// so every surface's root is its lowest group and the numbering is the same whatever
// order the hooks land in.
#include <cmath>
#include <cstring>

#include "nimbus_host.hpp"

namespace nb {
namespace {

struct SegP {
  double flat_max, spread_min, cos_join, join_dist, cos_edge;
  int min_points, edge_min_groups;
};

// Per group (subvoxel) results, structure of arrays.
struct Groups {
  double* cen;      // [G*3] centroid
  double* nor;      // [G*3] plane normal, oriented by the input normals
  double* cov;      // [G*6] covariance xx xy xz yy yz zz
  uint32_t* cnt;    // points
  int32_t* gs;      // [G*3] subvoxel coordinates
  uint8_t* planar;
};

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations: on return
// w holds the eigenvalues and the columns of v the eigenvectors.
__device__ void jacobi3(double a[3][3], double w[3], double v[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double scale = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off == 0.0 || off <= 1e-36 * scale) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
      if (a[p][q] == 0.0) continue;
      const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
      const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      for (int k = 0; k < 3; ++k) {
        const double akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        const double apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        const double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  for (int i = 0; i < 3; ++i) w[i] = a[i][i];
}

// Order of the eigenvalues: i0 smallest, i1 middle, i2 largest.
__device__ __forceinline__ void order3(const double w[3], int& i0, int& i1, int& i2) {
  i0 = 0;
  if (w[1] < w[i0]) i0 = 1;
  if (w[2] < w[i0]) i0 = 2;
  i2 = 0;
  if (w[1] > w[i2]) i2 = 1;
  if (w[2] > w[i2]) i2 = 2;
  if (i2 == i0) i2 = (i0 + 1) % 3;
  i1 = 3 - i0 - i2;
}

// Plane of each group: FP64 centroid and covariance in two passes over its points in
// input order, the eigenvector of the smallest eigenvalue turned to agree with the
// sum of the input normals, and the planarity test.
__global__ void k_seg_fit(DScene d, SegP sp, Groups G, int64_t n_groups) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const IERec r = d.ies[g];
  const uint32_t pb = __float_as_uint(r.bbc_pb.w), pc = __float_as_uint(r.sc_pc.w);
  double s[3] = {0.0, 0.0, 0.0}, ns[3] = {0.0, 0.0, 0.0};
  for (uint32_t k = 0; k < pc; ++k) {
    const float4 P = d.pts[pb + k], N = d.pnrm[pb + k];
    s[0] += (double)P.x; s[1] += (double)P.y; s[2] += (double)P.z;
    ns[0] += (double)N.x; ns[1] += (double)N.y; ns[2] += (double)N.z;
  }
  const double m = (double)pc;
  const double c[3] = {s[0] / m, s[1] / m, s[2] / m};
  double cxx = 0, cxy = 0, cxz = 0, cyy = 0, cyz = 0, czz = 0;
  for (uint32_t k = 0; k < pc; ++k) {
    const float4 P = d.pts[pb + k];
    const double dx = (double)P.x - c[0], dy = (double)P.y - c[1], dz = (double)P.z - c[2];
    cxx += dx * dx; cxy += dx * dy; cxz += dx * dz;
    cyy += dy * dy; cyz += dy * dz; czz += dz * dz;
  }
  double a[3][3] = {{cxx / m, cxy / m, cxz / m}, {cxy / m, cyy / m, cyz / m}, {cxz / m, cyz / m, czz / m}};
  const double cov[6] = {a[0][0], a[0][1], a[0][2], a[1][1], a[1][2], a[2][2]};
  const double tr = a[0][0] + a[1][1] + a[2][2];
  double w[3], v[3][3];
  jacobi3(a, w, v);
  int i0, i1, i2;
  order3(w, i0, i1, i2);
  double n[3] = {v[0][i0], v[1][i0], v[2][i0]};
  if (dot3(n, ns) < 0.0) {
    n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
  }
  const bool planar = (int)pc >= sp.min_points && tr > 0.0 && w[i0] <= sp.flat_max * tr && w[i1] >= sp.spread_min * tr;
  for (int i = 0; i < 3; ++i) {
    G.cen[3 * g + i] = c[i];
    G.nor[3 * g + i] = n[i];
  }
  for (int i = 0; i < 6; ++i) G.cov[6 * g + i] = cov[i];
  G.cnt[g] = pc;
  G.planar[g] = planar ? 1 : 0;
  // subvoxel of the group from its centre, o + (gs + 1/2) h_s
  const double o[3] = {d.odx, d.ody, d.odz};
  const float sc[3] = {r.sc_pc.x, r.sc_pc.y, r.sc_pc.z};
  for (int i = 0; i < 3; ++i) G.gs[3 * g + i] = (int)floor(((double)sc[i] - o[i]) / d.hsd);
}

// Group of subvoxel (x, y, z), or -1: the voxel's IEs are the groups of its subvoxels.
__device__ int find_group(const DScene& d, const int32_t* gs, int x, int y, int z) {
  const int dv = d.dv;
  if (x < 0 || y < 0 || z < 0 || x >= d.nx * dv || y >= d.ny * dv || z >= d.nz * dv) return -1;
  const uint2 cell = d.cells[cell_index(d, x / dv, y / dv, z / dv)];
  for (uint32_t k = 0; k < cell.y; ++k) {
    const int g = (int)(cell.x + k);
    if (gs[3 * g] == x && gs[3 * g + 1] == y && gs[3 * g + 2] == z) return g;
  }
  return -1;
}

// The 26 neighbours of group g, in (dz, dy, dx) loop order; returns how many exist.
__device__ int neighbours(const DScene& d, const int32_t* gs, int64_t g, int out[26]) {
  const int x = gs[3 * g], y = gs[3 * g + 1], z = gs[3 * g + 2];
  int m = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0 && dz == 0) continue;
        const int h = find_group(d, gs, x + dx, y + dy, z + dz);
        if (h >= 0) out[m++] = h;
      }
  return m;
}

__device__ __forceinline__ bool joined(const Groups& G, const SegP& sp, int a, int b) {
  const double* na = G.nor + 3 * a;
  const double* nb = G.nor + 3 * b;
  const double dab[3] = {G.cen[3 * b] - G.cen[3 * a], G.cen[3 * b + 1] - G.cen[3 * a + 1], G.cen[3 * b + 2] - G.cen[3 * a + 2]};
  const double dba[3] = {-dab[0], -dab[1], -dab[2]};
  return dot3(na, nb) >= sp.cos_join && fabs(dot3(na, dab)) <= sp.join_dist && fabs(dot3(nb, dba)) <= sp.join_dist;
}

// Root of x (every chain ends at a root within n steps); -1 if the bound is hit.
__device__ int uf_find(const volatile int* parent, int x, int64_t n) {
  for (int64_t i = 0; i <= n; ++i) {
    const int p = parent[x];
    if (p == x) return x;
    x = p;
  }
  return -1;
}

// Join the sets of a and b: the larger root is hooked under the smaller one with a
// compare-and-swap; a failed swap means that root was hooked meanwhile, so retry.
__device__ void uf_union(int* parent, int a, int b, int64_t n, uint32_t* err) {
  for (int it = 0; it < (1 << 20); ++it) {
    int ra = uf_find(parent, a, n), rb = uf_find(parent, b, n);
    if (ra < 0 || rb < 0) {
      atomicOr(err, 1u);
      return;
    }
    if (ra == rb) return;
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    if (atomicCAS(&parent[rb], rb, ra) == rb) return;
  }
  atomicOr(err, 2u);
}

__global__ void k_seg_init(int* parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    parent[i] = (int)i;
}

__global__ void k_seg_link(DScene d, SegP sp, Groups G, int64_t n, int* parent, uint32_t* err) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n || !G.planar[a]) return;
  int nb[26];
  const int m = neighbours(d, G.gs, a, nb);
  for (int j = 0; j < m; ++j) {
    const int b = nb[j];
    if (b > a && G.planar[b] && joined(G, sp, (int)a, b)) uf_union(parent, (int)a, b, n, err);
  }
}

__global__ void k_seg_roots(const int* parent, int64_t n, int* root, uint32_t* is_root, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = uf_find(parent, (int)i, n);
    if (r < 0) atomicOr(err, 1u);
    root[i] = r < 0 ? (int)i : r;
    is_root[i] = root[i] == (int)i ? 1u : 0u;
  }
}

__global__ void k_seg_sid(const int* root, const uint32_t* pos, int64_t n, uint32_t* sid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sid[i] = pos[root[i]];
}

__device__ __forceinline__ bool fits(const Groups& G, const SegP& sp, int h, const double P[3], const double N[3]) {
  if (!G.planar[h]) return false;
  const double* nh = G.nor + 3 * h;
  const double dp[3] = {P[0] - G.cen[3 * h], P[1] - G.cen[3 * h + 1], P[2] - G.cen[3 * h + 2]};
  return dot3(nh, N) >= sp.cos_join && fabs(dot3(nh, dp)) <= sp.join_dist;
}

// Point labels: a point keeps its group's surface when the group fits it, else takes
// the nearest fitting planar neighbour's (ties: the lower group), else its own.
__global__ void k_seg_labels(DScene d, SegP sp, Groups G, int64_t n_groups, const uint32_t* sid, uint32_t* labels) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  int nb[26];
  int m = neighbours(d, G.gs, g, nb);
  int k = 0;
  for (int j = 0; j < m; ++j)
    if (G.planar[nb[j]]) nb[k++] = nb[j];
  m = k;
  for (int i = 1; i < m; ++i) {   // ascending group order
    const int x = nb[i];
    int j = i - 1;
    while (j >= 0 && nb[j] > x) {
      nb[j + 1] = nb[j];
      --j;
    }
    nb[j + 1] = x;
  }
  const IERec r = d.ies[g];
  const uint32_t pb = __float_as_uint(r.bbc_pb.w), pc = __float_as_uint(r.sc_pc.w);
  for (uint32_t q = 0; q < pc; ++q) {
    const float4 Pf = d.pts[pb + q], Nf = d.pnrm[pb + q];
    const double P[3] = {(double)Pf.x, (double)Pf.y, (double)Pf.z};
    const double N[3] = {(double)Nf.x, (double)Nf.y, (double)Nf.z};
    uint32_t lab = sid[g];
    if (!fits(G, sp, (int)g, P, N)) {
      int best = -1;
      double bd = 0.0;
      for (int j = 0; j < m; ++j) {
        const int h = nb[j];
        if (!fits(G, sp, h, P, N)) continue;
        const double dp[3] = {P[0] - G.cen[3 * h], P[1] - G.cen[3 * h + 1], P[2] - G.cen[3 * h + 2]};
        const double dist = fabs(dot3(G.nor + 3 * h, dp));
        if (best < 0 || dist < bd) {
          best = h;
          bd = dist;
        }
      }
      if (best >= 0) lab = sid[best];
    }
    labels[__float_as_uint(Pf.w)] = lab;   // w holds the point's input index
  }
}

__global__ void k_seg_planar_keys(const Groups G, const uint32_t* sid, int64_t n, const uint32_t* pos,
                                  uint64_t* keys, uint32_t* vals) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (G.planar[g]) {
      keys[pos[g]] = sid[g];
      vals[pos[g]] = (uint32_t)g;
    }
}

__global__ void k_run_starts(const uint64_t* keys, int64_t n, uint32_t* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_run_index(const uint32_t* flags, const uint32_t* pos, int64_t n, uint32_t* first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) first[pos[i]] = (uint32_t)i;
}

// Plane of each surface from the pooled moments of its planar groups (in group order):
// the centroid, the scatter about it, the normal turned to agree with the groups'.
__global__ void k_seg_surfaces(Groups G, const uint64_t* keys, const uint32_t* vals, const uint32_t* first,
                               int64_t n_runs, int64_t n_planar, double* sc, double* sn, uint32_t* sgroups) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_runs) return;
  const uint32_t b = first[r], e = r + 1 < n_runs ? first[r + 1] : (uint32_t)n_planar;
  const uint32_t s = (uint32_t)keys[b];
  double m = 0.0, c[3] = {0.0, 0.0, 0.0}, ns[3] = {0.0, 0.0, 0.0};
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t g = vals[i];
    const double k = (double)G.cnt[g];
    m += k;
    for (int a = 0; a < 3; ++a) {
      c[a] += k * G.cen[3 * g + a];
      ns[a] += G.nor[3 * g + a];
    }
  }
  for (int a = 0; a < 3; ++a) c[a] /= m;
  double S[6] = {0, 0, 0, 0, 0, 0};
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t g = vals[i];
    const double k = (double)G.cnt[g];
    const double d0 = G.cen[3 * g] - c[0], d1 = G.cen[3 * g + 1] - c[1], d2 = G.cen[3 * g + 2] - c[2];
    const double* C = G.cov + 6 * g;
    S[0] += k * (C[0] + d0 * d0); S[1] += k * (C[1] + d0 * d1); S[2] += k * (C[2] + d0 * d2);
    S[3] += k * (C[3] + d1 * d1); S[4] += k * (C[4] + d1 * d2); S[5] += k * (C[5] + d2 * d2);
  }
  double a[3][3] = {{S[0] / m, S[1] / m, S[2] / m}, {S[1] / m, S[3] / m, S[4] / m}, {S[2] / m, S[4] / m, S[5] / m}};
  double w[3], v[3][3];
  jacobi3(a, w, v);
  int i0, i1, i2;
  order3(w, i0, i1, i2);
  double n[3] = {v[0][i0], v[1][i0], v[2][i0]};
  if (dot3(n, ns) < 0.0) {
    n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
  }
  for (int k = 0; k < 3; ++k) {
    sc[3 * s + k] = c[k];
    sn[3 * s + k] = n[k];
  }
  sgroups[s] = e - b;
}

// Meeting groups: for planar a and planar neighbour b > a on another surface, the pair
// of surfaces (A < B) gets both groups.  Counted, then written at scanned offsets.
__global__ void k_seg_meet(DScene d, Groups G, const uint32_t* sid, int64_t n, const uint32_t* off, uint32_t* count,
                           uint64_t* keys, uint32_t* vals) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  uint32_t c = 0;
  if (G.planar[a]) {
    int nb[26];
    const int m = neighbours(d, G.gs, a, nb);
    for (int j = 0; j < m; ++j) {
      const int b = nb[j];
      if (b <= a || !G.planar[b] || sid[a] == sid[b]) continue;
      if (keys) {
        const uint64_t A = min(sid[a], sid[b]), B = max(sid[a], sid[b]);
        const uint64_t key = (A << 32) | B;
        keys[off[a] + c] = key;
        vals[off[a] + c] = (uint32_t)a;
        keys[off[a] + c + 1] = key;
        vals[off[a] + c + 1] = (uint32_t)b;
      }
      c += 2;
    }
  }
  if (count) count[a] = c;
}

__global__ void k_seg_gather_keys(const uint64_t* key_of_entry, const uint32_t* entry, int64_t n, uint64_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = key_of_entry[entry[i]];
}

__global__ void k_seg_u32_to_u64(const uint32_t* in, int64_t n, uint64_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

__global__ void k_iota(uint32_t* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

// Distinct (pair, group) entries: the first of each run of equal ones.
__global__ void k_seg_unique(const uint64_t* keys, const uint32_t* vals, int64_t n, uint32_t* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1] || vals[i] != vals[i - 1]) ? 1u : 0u;
}

__global__ void k_seg_compact(const uint64_t* keys, const uint32_t* vals, const uint32_t* flags, const uint32_t* pos,
                              int64_t n, uint64_t* ok, uint32_t* ov) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) {
      ok[pos[i]] = keys[i];
      ov[pos[i]] = vals[i];
    }
}

// One thread per meeting pair of surfaces: the exterior-edge test and the edge.
__global__ void k_seg_edges(Groups G, SegP sp, const uint64_t* keys, const uint32_t* vals, const uint32_t* first,
                            int64_t n_pairs, int64_t n_entries, const double* sc, const double* sn,
                            const uint32_t* sgroups, uint32_t* ok, double* edges) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  const uint32_t b = first[p], e = p + 1 < n_pairs ? first[p + 1] : (uint32_t)n_entries;
  const uint32_t A = (uint32_t)(keys[b] >> 32), B = (uint32_t)(keys[b] & 0xffffffffu);
  ok[p] = 0;
  if ((int)sgroups[A] < sp.edge_min_groups || (int)sgroups[B] < sp.edge_min_groups) return;
  const double* cA = sc + 3 * A;
  const double* cB = sc + 3 * B;
  const double* nA = sn + 3 * A;
  const double* nB = sn + 3 * B;
  const double dBA[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};
  const double dAB[3] = {-dBA[0], -dBA[1], -dBA[2]};
  if (!(dot3(nA, nB) <= sp.cos_edge && dot3(nA, dBA) < 0.0 && dot3(nB, dAB) < 0.0)) return;
  double mid[3] = {0.0, 0.0, 0.0};
  for (uint32_t i = b; i < e; ++i)
    for (int a = 0; a < 3; ++a) mid[a] += G.cen[3 * vals[i] + a];
  for (int a = 0; a < 3; ++a) mid[a] /= (double)(e - b);
  double w[3] = {nA[1] * nB[2] - nA[2] * nB[1], nA[2] * nB[0] - nA[0] * nB[2], nA[0] * nB[1] - nA[1] * nB[0]};
  const double wl = sqrt(dot3(w, w));
  for (int a = 0; a < 3; ++a) w[a] /= wl;
  // the point of both planes nearest mid: mid + al nA + be nB (2x2 normal equations)
  const double m00 = dot3(nA, nA), m01 = dot3(nA, nB), m11 = dot3(nB, nB);
  const double r0 = dot3(nA, cA) - dot3(nA, mid), r1 = dot3(nB, cB) - dot3(nB, mid);
  const double det = m00 * m11 - m01 * m01;
  const double al = (r0 * m11 - r1 * m01) / det, be = (m00 * r1 - m01 * r0) / det;
  double x0[3];
  for (int a = 0; a < 3; ++a) x0[a] = mid[a] + al * nA[a] + be * nB[a];
  double tmin = 0.0, tmax = 0.0;
  for (uint32_t i = b; i < e; ++i) {
    const double* c = G.cen + 3 * vals[i];
    const double dc[3] = {c[0] - x0[0], c[1] - x0[1], c[2] - x0[2]};
    const double t = dot3(w, dc);
    if (i == b || t < tmin) tmin = t;
    if (i == b || t > tmax) tmax = t;
  }
  double* E = edges + 12 * p;
  for (int a = 0; a < 3; ++a) {
    E[a] = x0[a] + tmin * w[a];
    E[3 + a] = x0[a] + tmax * w[a];
    E[6 + a] = nA[a];
    E[9 + a] = nB[a];
  }
  ok[p] = 1;
}

__global__ void k_seg_edges_out(const double* edges, const uint32_t* ok, const uint32_t* pos, int64_t n_pairs,
                                int64_t cap, uint32_t label0, double* out, uint32_t* out_label) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs; p += (int64_t)gridDim.x * blockDim.x)
    if (ok[p] && pos[p] < cap) {
      for (int a = 0; a < 12; ++a) out[12 * (int64_t)pos[p] + a] = edges[12 * p + a];
      out_label[pos[p]] = label0 + pos[p];
    }
}

__global__ void k_seg_planar_flags(Groups G, int64_t n, uint32_t* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = G.planar[i];
}

__global__ void k_seg_gather_u32(const uint32_t* src, const uint32_t* idx, int64_t n, uint32_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = src[idx[i]];
}

unsigned g_for(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + b - 1) / b, 1 << 20)); }

// Reads a device count back to the host.
int read_u32(std::string* err, const uint32_t* d, uint32_t* h, cudaStream_t st) {
  NB_CUDA(err, cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  return NIMBUS_OK;
}

// Runs of equal keys in sorted keys[n]: first[r] = start of run r; returns the count.
int key_runs(Scratch& sc, const uint64_t* keys, int64_t n, uint32_t** first, uint32_t* n_runs, cudaStream_t st) {
  std::string* err = sc.mem->err;
  uint32_t *flags, *pos, *tot;
  NB_TRY(sc.get(&flags, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&pos, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(first, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&tot, 1));
  k_run_starts<<<g_for(n, 256), 256, 0, st>>>(keys, n, flags);
  NB_LAUNCHED(err);
  NB_TRY(exclusive_scan(sc, flags, pos, n, tot));
  k_run_index<<<g_for(n, 256), 256, 0, st>>>(flags, pos, n, *first);
  NB_LAUNCHED(err);
  return read_u32(err, tot, n_runs, st);
}

}  // namespace

int segment_scene(Mem& mem, SceneObj* S, const nimbus_segment_params* p, uint32_t* labels_out, double* edges_out,
                  uint32_t* edge_labels_out, int64_t edges_cap, nimbus_segment_counts* counts, cudaStream_t st) {
  std::string* err = mem.err;
  const DScene& d = S->d;
  const int64_t G = S->n_ie, n = S->n_points;
  std::memset(counts, 0, sizeof *counts);
  SegP sp;
  sp.flat_max = p->flat_max;
  sp.spread_min = p->spread_min;
  sp.cos_join = std::cos(p->join_angle);
  sp.join_dist = p->join_dist;
  sp.cos_edge = std::cos(p->edge_angle);
  sp.min_points = p->min_points;
  sp.edge_min_groups = p->edge_min_groups;
  if (G >= (1ll << 31)) {
    *err = "segment: too many subvoxel groups";
    return NIMBUS_ERR_ARG;
  }
  Scratch sc(&mem, st);
  StageTimer tm(st);
  const int e0 = tm.mark();
  Groups gr;
  uint32_t *labels, *err_d, *is_root, *pos, *sid, *tot, *pflag, *ppos;
  int *parent, *root;
  const int64_t G1 = std::max<int64_t>(1, G);
  NB_TRY(sc.get(&gr.cen, 3 * G1));
  NB_TRY(sc.get(&gr.nor, 3 * G1));
  NB_TRY(sc.get(&gr.cov, 6 * G1));
  NB_TRY(sc.get(&gr.cnt, G1));
  NB_TRY(sc.get(&gr.gs, 3 * G1));
  NB_TRY(sc.get(&gr.planar, G1));
  NB_TRY(sc.get(&labels, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&err_d, 1));
  NB_TRY(sc.get(&parent, G1));
  NB_TRY(sc.get(&root, G1));
  NB_TRY(sc.get(&is_root, G1));
  NB_TRY(sc.get(&pos, G1));
  NB_TRY(sc.get(&sid, G1));
  NB_TRY(sc.get(&pflag, G1));
  NB_TRY(sc.get(&ppos, G1));
  NB_TRY(sc.get(&tot, 2));
  NB_CUDA(err, cudaMemsetAsync(err_d, 0, sizeof(uint32_t), st));
  NB_CUDA(err, cudaMemsetAsync(tot, 0, 2 * sizeof(uint32_t), st));
  if (G > 0) {
    // steps 2-4: group planes, surfaces, point labels
    k_seg_fit<<<g_for(G, 128), 128, 0, st>>>(d, sp, gr, G);
    NB_LAUNCHED(err);
    k_seg_init<<<g_for(G, 256), 256, 0, st>>>(parent, G);
    NB_LAUNCHED(err);
    k_seg_link<<<g_for(G, 128), 128, 0, st>>>(d, sp, gr, G, parent, err_d);
    NB_LAUNCHED(err);
    k_seg_roots<<<g_for(G, 256), 256, 0, st>>>(parent, G, root, is_root, err_d);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(sc, is_root, pos, G, tot));
    k_seg_sid<<<g_for(G, 256), 256, 0, st>>>(root, pos, G, sid);
    NB_LAUNCHED(err);
    k_seg_labels<<<g_for(G, 128), 128, 0, st>>>(d, sp, gr, G, sid, labels);
    NB_LAUNCHED(err);
    k_seg_planar_flags<<<g_for(G, 256), 256, 0, st>>>(gr, G, pflag);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(sc, pflag, ppos, G, tot + 1));
  }
  uint32_t h_tot[2] = {0, 0}, h_err = 0;
  NB_CUDA(err, cudaMemcpyAsync(h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaMemcpyAsync(&h_err, err_d, sizeof h_err, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  if (h_err) {
    *err = "segment: union-find step bound reached";
    return NIMBUS_ERR_TIMEOUT;
  }
  const int64_t n_surf = h_tot[0], n_planar = h_tot[1];
  int64_t n_edges = 0;
  if (n_planar > 0) {
    // step 5: surface planes from their planar groups, in group order
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt, *first, n_runs = 0;
    NB_TRY(sc.get(&keys, n_planar));
    NB_TRY(sc.get(&keys_alt, n_planar));
    NB_TRY(sc.get(&vals, n_planar));
    NB_TRY(sc.get(&vals_alt, n_planar));
    k_seg_planar_keys<<<g_for(G, 256), 256, 0, st>>>(gr, sid, G, ppos, keys, vals);
    NB_LAUNCHED(err);
    NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, n_planar, bits_for((uint64_t)n_surf)));
    NB_TRY(key_runs(sc, keys, n_planar, &first, &n_runs, st));
    double *scen, *snor;
    uint32_t* sgroups;
    NB_TRY(sc.get(&scen, 3 * n_surf));
    NB_TRY(sc.get(&snor, 3 * n_surf));
    NB_TRY(sc.get(&sgroups, n_surf));
    NB_CUDA(err, cudaMemsetAsync(sgroups, 0, n_surf * sizeof(uint32_t), st));
    k_seg_surfaces<<<g_for(n_runs, 64), 64, 0, st>>>(gr, keys, vals, first, n_runs, n_planar, scen, snor, sgroups);
    NB_LAUNCHED(err);
    // groups where two surfaces meet: counted, then written at scanned offsets
    uint32_t *mcount, *moff, *mtot, n_ent = 0;
    NB_TRY(sc.get(&mcount, G));
    NB_TRY(sc.get(&moff, G));
    NB_TRY(sc.get(&mtot, 1));
    k_seg_meet<<<g_for(G, 128), 128, 0, st>>>(d, gr, sid, G, nullptr, mcount, nullptr, nullptr);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(sc, mcount, moff, G, mtot));
    NB_TRY(read_u32(err, mtot, &n_ent, st));
    if (n_ent > 0) {
      uint64_t *ek, *gk, *gk_alt, *pk, *pk_alt, *uk;
      uint32_t *ev, *idx, *idx_alt, *pv, *pv_alt, *uflag, *upos, *uv, *utot, n_u = 0;
      NB_TRY(sc.get(&ek, n_ent));
      NB_TRY(sc.get(&ev, n_ent));
      k_seg_meet<<<g_for(G, 128), 128, 0, st>>>(d, gr, sid, G, moff, nullptr, ek, ev);
      NB_LAUNCHED(err);
      // order the entries by (pair, group): by group first, then stably by pair
      NB_TRY(sc.get(&gk, n_ent));
      NB_TRY(sc.get(&gk_alt, n_ent));
      NB_TRY(sc.get(&idx, n_ent));
      NB_TRY(sc.get(&idx_alt, n_ent));
      k_seg_u32_to_u64<<<g_for(n_ent, 256), 256, 0, st>>>(ev, n_ent, gk);
      NB_LAUNCHED(err);
      k_iota<<<g_for(n_ent, 256), 256, 0, st>>>(idx, n_ent);
      NB_LAUNCHED(err);
      NB_TRY(radix_sort(sc, gk, idx, gk_alt, idx_alt, n_ent, bits_for((uint64_t)G)));
      NB_TRY(sc.get(&pk, n_ent));
      NB_TRY(sc.get(&pk_alt, n_ent));
      NB_TRY(sc.get(&pv, n_ent));
      NB_TRY(sc.get(&pv_alt, n_ent));
      k_seg_gather_keys<<<g_for(n_ent, 256), 256, 0, st>>>(ek, idx, n_ent, pk);
      NB_LAUNCHED(err);
      k_seg_gather_u32<<<g_for(n_ent, 256), 256, 0, st>>>(ev, idx, n_ent, pv);
      NB_LAUNCHED(err);
      NB_TRY(radix_sort(sc, pk, pv, pk_alt, pv_alt, n_ent, 32 + bits_for((uint64_t)n_surf)));
      NB_TRY(sc.get(&uflag, n_ent));
      NB_TRY(sc.get(&upos, n_ent));
      NB_TRY(sc.get(&uk, n_ent));
      NB_TRY(sc.get(&uv, n_ent));
      NB_TRY(sc.get(&utot, 1));
      k_seg_unique<<<g_for(n_ent, 256), 256, 0, st>>>(pk, pv, n_ent, uflag);
      NB_LAUNCHED(err);
      NB_TRY(exclusive_scan(sc, uflag, upos, n_ent, utot));
      k_seg_compact<<<g_for(n_ent, 256), 256, 0, st>>>(pk, pv, uflag, upos, n_ent, uk, uv);
      NB_LAUNCHED(err);
      NB_TRY(read_u32(err, utot, &n_u, st));
      uint32_t *pfirst, n_pairs = 0;
      NB_TRY(key_runs(sc, uk, n_u, &pfirst, &n_pairs, st));
      // step 5: the exterior-edge test per pair of meeting surfaces
      double* etmp;
      uint32_t *eok, *epos, *etot, h_edges = 0;
      NB_TRY(sc.get(&etmp, 12 * (int64_t)n_pairs));
      NB_TRY(sc.get(&eok, n_pairs));
      NB_TRY(sc.get(&epos, n_pairs));
      NB_TRY(sc.get(&etot, 1));
      k_seg_edges<<<g_for(n_pairs, 64), 64, 0, st>>>(gr, sp, uk, uv, pfirst, n_pairs, n_u, scen, snor, sgroups, eok,
                                                     etmp);
      NB_LAUNCHED(err);
      NB_TRY(exclusive_scan(sc, eok, epos, n_pairs, etot));
      NB_TRY(read_u32(err, etot, &h_edges, st));
      n_edges = h_edges;
      const int64_t n_out = std::min<int64_t>(n_edges, edges_cap);
      if (n_out > 0) {
        double* eout;
        uint32_t* elab;
        NB_TRY(sc.get(&eout, 12 * n_out));
        NB_TRY(sc.get(&elab, n_out));
        k_seg_edges_out<<<g_for(n_pairs, 128), 128, 0, st>>>(etmp, eok, epos, n_pairs, n_out, (uint32_t)n_surf, eout,
                                                             elab);
        NB_LAUNCHED(err);
        NB_CUDA(err, cudaMemcpyAsync(edges_out, eout, 12 * n_out * sizeof(double), cudaMemcpyDefault, st));
        NB_CUDA(err, cudaMemcpyAsync(edge_labels_out, elab, n_out * sizeof(uint32_t), cudaMemcpyDefault, st));
      }
    }
  }
  if (n > 0) NB_CUDA(err, cudaMemcpyAsync(labels_out, labels, n * sizeof(uint32_t), cudaMemcpyDefault, st));
  const int e1 = tm.mark();
  NB_CUDA(err, cudaStreamSynchronize(st));
  counts->n_groups = G;
  counts->n_planar = n_planar;
  counts->n_surfaces = n_surf;
  counts->n_edges = n_edges;
  counts->ms = tm.ms(e0, e1);
  if (n_edges > edges_cap) {
    *err = "segment: more exterior edges than edges_cap (see n_edges)";
    return NIMBUS_ERR_OVERFLOW;
  }
  return NIMBUS_OK;
}

}  // namespace nb
