// Voxelisation (Section 2.1): labelled point cloud + edges -> intersectable
// entities (IEs) per subvoxel, per-voxel IE ranges and the march distance field
// of voxel cone tracing (Section 2.2.4).
//
// B300 design: a 64-bit sort key per point, (voxel, subvoxel, kind, label), packed
// so that one stable radix sort groups every subvoxel's points by label and orders
// the groups by voxel; then one thread per IE reduces its contiguous run, and two
// passes over the IE table give each voxel its IE range.  Edge segments join the
// same sort with the kind bit set, so edge IEs sit in their voxel's range.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>
#include <mutex>

#include "nimbus_host.hpp"

namespace nb {

namespace {

constexpr uint64_t INVALID_KEY = ~0ull;

struct GridK {
  float o[3];
  float hs;
  int gmax[3];        // largest global subvoxel index per axis
  int dv, nx, ny;
  int sub_bits, id_bits;
};

__device__ __forceinline__ uint32_t f2o(float f) {  // order-preserving float -> uint
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_bounds(const float* __restrict__ xyz, const uint32_t* __restrict__ label, int64_t n,
                         uint32_t* __restrict__ out /* lo[3] hi[3] maxlabel */) {
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  uint32_t ml = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float v = xyz[3 * i + a];
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
    ml = max(ml, label[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
    ml = max(ml, __shfl_xor_sync(0xffffffffu, ml, o));
  }
  if ((threadIdx.x & 31) == 0) {
    for (int a = 0; a < 3; ++a) {
      atomicMin(&out[a], f2o(lo[a]));
      atomicMax(&out[3 + a], f2o(hi[a]));
    }
    atomicMax(&out[6], ml);
  }
}

__device__ __forceinline__ uint64_t pack_key(const GridK& g, const int gs[3], uint32_t kind, uint32_t id) {
  const int dv = g.dv;
  uint64_t cell = ((uint64_t)(gs[2] / dv) * g.ny + (gs[1] / dv)) * g.nx + (gs[0] / dv);
  uint64_t sub = (uint64_t)(((gs[2] % dv) * dv + (gs[1] % dv)) * dv + (gs[0] % dv));
  return (cell << (g.sub_bits + 1 + g.id_bits)) | (sub << (1 + g.id_bits)) | ((uint64_t)kind << g.id_bits) |
         (uint64_t)id;
}

__global__ void k_point_keys(GridK g, const float* __restrict__ xyz, const uint32_t* __restrict__ label, int64_t n,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int gs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) gs[a] = subvoxel_axis(xyz[3 * i + a], g.o[a], g.hs, g.gmax[a]);
    keys[i] = pack_key(g, gs, IE_POINT, label[i]);
    vals[i] = (uint32_t)i;
  }
}

// One thread per edge: the edge is cut into nf fine pieces; a piece belongs to the
// subvoxel of its midpoint (FP64 midpoint, rounded to FP32, binned like a point),
// and runs of pieces in one subvoxel form one edge IE.  Slots of the edge's range
// left over get the invalid key.  FP64 operations are explicitly rounded so the
// pieces match any IEEE implementation that performs the same steps.
__global__ void k_edge_pieces(GridK g, const double* __restrict__ edges, int n_edges,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ nf_arr, int64_t n_points,
                              uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, int4* __restrict__ pieces,
                              uint32_t* __restrict__ n_valid) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_edges) return;
  const double* E = edges + 12 * e;
  const double d[3] = {__dsub_rn(E[3], E[0]), __dsub_rn(E[4], E[1]), __dsub_rn(E[5], E[2])};
  const int nf = nf_arr[e];
  const int64_t base = off[e];
  int64_t slot = base;
  int prev[3] = {-1, -1, -1};
  int i0 = 0;
  for (int i = 0; i <= nf; ++i) {
    int gs[3] = {-2, -2, -2};
    if (i < nf) {
      double f = __ddiv_rn((double)i + 0.5, (double)nf);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double m = __dadd_rn(E[a], __dmul_rn(f, d[a]));
        gs[a] = subvoxel_axis(__double2float_rn(m), g.o[a], g.hs, g.gmax[a]);
      }
    }
    bool change = (i == nf) || gs[0] != prev[0] || gs[1] != prev[1] || gs[2] != prev[2];
    if (change && i > 0) {  // close the run [i0, i-1] held in prev
      keys[n_points + slot] = pack_key(g, prev, IE_EDGE, (uint32_t)e);
      vals[n_points + slot] = (uint32_t)(n_points + slot);
      pieces[slot - 0] = make_int4(e, i0, i - 1, nf);
      ++slot;
    }
    if (change) {
      i0 = i;
      prev[0] = gs[0]; prev[1] = gs[1]; prev[2] = gs[2];
    }
  }
  atomicAdd(n_valid, (uint32_t)(slot - base));
  for (int64_t s2 = slot; s2 < base + nf; ++s2) {
    keys[n_points + s2] = INVALID_KEY;
    vals[n_points + s2] = (uint32_t)(n_points + s2);
  }
}

__global__ void k_run_flags(const uint64_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    flags[i] = (k != INVALID_KEY && (i == 0 || k != keys[i - 1])) ? 1u : 0u;
  }
}

__global__ void k_run_starts(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ ids, int64_t n,
                             uint32_t* __restrict__ starts, uint32_t n_ie, uint32_t n_valid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) starts[ids[i]] = (uint32_t)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) starts[n_ie] = n_valid;
}

__global__ void k_gather(const uint32_t* __restrict__ vals, int64_t n_valid, int64_t n_points,
                         const float* __restrict__ xyz, const float* __restrict__ nrm, float4* __restrict__ pts,
                         float4* __restrict__ pnrm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_valid;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = vals[i];
    if (v < n_points) {
      pts[i] = make_float4(xyz[3 * (int64_t)v], xyz[3 * (int64_t)v + 1], xyz[3 * (int64_t)v + 2], __uint_as_float(v));
      pnrm[i] = make_float4(nrm[3 * (int64_t)v], nrm[3 * (int64_t)v + 1], nrm[3 * (int64_t)v + 2], 0.f);
    } else {
      pts[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      pnrm[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

struct BuildK {
  GridK g;
  double o[3], hs;
  int64_t n_points;
  int n_ie;
};

// One thread per IE: reduce its run of sorted entries into the IE record.  Point
// IE: reception point = centroid, normal = normalised mean normal, bounding-box
// centre, material = smallest in the group.  Edge IE: reception point = midpoint
// of its piece range on the edge.
__global__ void k_ie_build(BuildK b, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                           const uint32_t* __restrict__ starts, const float4* __restrict__ pts,
                           const float4* __restrict__ pnrm, const uint8_t* __restrict__ material,
                           const int4* __restrict__ pieces, const double* __restrict__ edges,
                           IERec* __restrict__ ies, uint32_t* __restrict__ ie_cell) {
  int ie = blockIdx.x * blockDim.x + threadIdx.x;
  if (ie >= b.n_ie) return;
  const GridK& g = b.g;
  uint32_t s = starts[ie], e = starts[ie + 1];
  uint64_t key = keys[s];
  uint32_t id = (uint32_t)(key & ((1ull << g.id_bits) - 1));
  uint32_t kind = (uint32_t)((key >> g.id_bits) & 1ull);
  uint32_t sub = (uint32_t)((key >> (g.id_bits + 1)) & ((1ull << g.sub_bits) - 1));
  uint64_t cell = key >> (g.id_bits + 1 + g.sub_bits);
  const int dv = g.dv;
  int vx = (int)(cell % (uint64_t)g.nx), vy = (int)((cell / (uint64_t)g.nx) % (uint64_t)g.ny),
      vz = (int)(cell / ((uint64_t)g.nx * g.ny));
  int gs[3] = {vx * dv + (int)(sub % dv), vy * dv + (int)((sub / dv) % dv), vz * dv + (int)(sub / (dv * dv))};
  IERec r;
  float sc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) sc[a] = (float)(b.o[a] + ((double)gs[a] + 0.5) * b.hs);
  r.sc_pc = make_float4(sc[0], sc[1], sc[2], 0.f);
  if (kind == IE_POINT) {
    double sx = 0, sy = 0, sz = 0, nx_ = 0, ny_ = 0, nz_ = 0;
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    uint32_t mat = 255;
    for (uint32_t k = s; k < e; ++k) {
      float4 P = pts[k];
      float4 N = pnrm[k];
      sx = __dadd_rn(sx, (double)P.x); sy = __dadd_rn(sy, (double)P.y); sz = __dadd_rn(sz, (double)P.z);
      nx_ = __dadd_rn(nx_, (double)N.x); ny_ = __dadd_rn(ny_, (double)N.y); nz_ = __dadd_rn(nz_, (double)N.z);
      lo[0] = fminf(lo[0], P.x); lo[1] = fminf(lo[1], P.y); lo[2] = fminf(lo[2], P.z);
      hi[0] = fmaxf(hi[0], P.x); hi[1] = fmaxf(hi[1], P.y); hi[2] = fmaxf(hi[2], P.z);
      if (material) mat = min(mat, (uint32_t)material[vals[k]]);
      else mat = 0;
    }
    double inv = __drcp_rn((double)(e - s));
    double nn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(nx_, nx_), __dmul_rn(ny_, ny_)), __dmul_rn(nz_, nz_)));
    double ninv = nn > 0.0 ? __drcp_rn(nn) : 0.0;
    r.rp_lab = make_float4((float)__dmul_rn(inv, sx), (float)__dmul_rn(inv, sy), (float)__dmul_rn(inv, sz),
                           __uint_as_float(id));
    r.nrm_meta = make_float4((float)__dmul_rn(ninv, nx_), (float)__dmul_rn(ninv, ny_), (float)__dmul_rn(ninv, nz_),
                             __uint_as_float((uint32_t)IE_POINT | (mat << 8)));
    r.bbc_pb = make_float4((float)(0.5 * ((double)lo[0] + (double)hi[0])), (float)(0.5 * ((double)lo[1] + (double)hi[1])),
                           (float)(0.5 * ((double)lo[2] + (double)hi[2])), __uint_as_float(s));
    r.sc_pc.w = __uint_as_float(e - s);
    // bounds for the march test of the visibility rays (march_cannot_hit); a point
    // with a zero normal, or a zero mean normal, disables the test for this IE
    const float3 n0 = xyz(r.nrm_meta), cb = xyz(r.bbc_pb);
    float cmin = ninv > 0.0 ? 1.f : -1.f, dlo = 3.4e38f, dhi = -3.4e38f, rmax = 0.f;
    for (uint32_t k = s; k < e; ++k) {
      const float3 p = xyz(pts[k]) - cb, nk = xyz(pnrm[k]);
      const float nl = len(nk);
      cmin = fminf(cmin, nl > 0.f ? dot(nk, n0) / nl : -1.f);
      const float dd = dot(p, n0);
      dlo = fminf(dlo, dd);
      dhi = fmaxf(dhi, dd);
      rmax = fmaxf(rmax, len(p));
    }
    r.slab = make_float4(cmin - 1e-6f, dlo, dhi, rmax);
  } else {
    int4 pc = pieces[vals[s] - b.n_points];
    const double* E = edges + 12 * pc.x;
    double t0 = (double)pc.y / (double)pc.w, t1 = (double)(pc.z + 1) / (double)pc.w;
    double tm = 0.5 * (t0 + t1);
    float rp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rp[a] = (float)(E[a] + tm * (E[3 + a] - E[a]));
    float3 n = normalize(f3((float)(E[6] + E[9]), (float)(E[7] + E[10]), (float)(E[8] + E[11])));
    r.rp_lab = make_float4(rp[0], rp[1], rp[2], __uint_as_float(0u));  // label set on the host side below
    r.nrm_meta = make_float4(n.x, n.y, n.z, __uint_as_float((uint32_t)IE_EDGE | (255u << 8)));
    r.bbc_pb = make_float4(rp[0], rp[1], rp[2], __uint_as_float((uint32_t)pc.x));
    r.sc_pc.w = __uint_as_float(0u);
    r.slab = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  ies[ie] = r;
  ie_cell[ie] = (uint32_t)cell;
}

// Edge IEs carry their edge's label (looked up from the edge label table).
__global__ void k_edge_labels(IERec* __restrict__ ies, int n_ie, const uint32_t* __restrict__ edge_label) {
  int ie = blockIdx.x * blockDim.x + threadIdx.x;
  if (ie >= n_ie) return;
  float4 m = ies[ie].nrm_meta;
  if ((__float_as_uint(m.w) & 1u) == IE_EDGE) {
    uint32_t e = __float_as_uint(ies[ie].bbc_pb.w);
    ies[ie].rp_lab.w = __uint_as_float(edge_label[e]);
  }
}

__global__ void k_cell_begin(const uint32_t* __restrict__ ie_cell, int n_ie, uint2* __restrict__ cells) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ie) return;
  if (i == 0 || ie_cell[i] != ie_cell[i - 1]) cells[ie_cell[i]].x = (uint32_t)i;
}

__global__ void k_cell_count(const uint32_t* __restrict__ ie_cell, int n_ie, uint2* __restrict__ cells) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ie) return;
  if (i == n_ie - 1 || ie_cell[i] != ie_cell[i + 1]) {
    uint32_t c = ie_cell[i];
    cells[c].y = (uint32_t)i + 1u - cells[c].x;
  }
}

// March field, separable L-infinity distance transform (capped at 255):
// pass x gives the 1-D distance to the nearest voxel with IEs in each row; passes
// y and z take min over w of max(|v - w|, d(w)), which composes the L-infinity
// metric one axis at a time.  The scan over w stops once |v - w| reaches the best.
__global__ void k_march_x(const uint2* __restrict__ cells, int nx, int ny, int nz, uint8_t* __restrict__ d1) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= ny * nz) return;
  int64_t base = (int64_t)row * nx;
  int dist = 255;
  for (int x = 0; x < nx; ++x) {
    dist = cells[base + x].y > 0 ? 0 : min(dist + 1, 255);
    d1[base + x] = (uint8_t)dist;
  }
  dist = 255;
  for (int x = nx - 1; x >= 0; --x) {
    dist = cells[base + x].y > 0 ? 0 : min(dist + 1, 255);
    d1[base + x] = (uint8_t)min((int)d1[base + x], dist);
  }
}

__global__ void k_march_axis(const uint8_t* __restrict__ din, uint8_t* __restrict__ dout, int nx, int ny, int nz,
                             int axis) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)nx * ny * nz;
  if (i >= n) return;
  int y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
  int c = axis == 1 ? y : z;
  int lim = axis == 1 ? ny : nz;
  int64_t stride = axis == 1 ? nx : (int64_t)nx * ny;
  int best = din[i];
  for (int r = 1; r < best; ++r) {
    if (c - r >= 0) best = min(best, max(r, (int)din[i - r * stride]));
    if (c + r < lim) best = min(best, max(r, (int)din[i + r * stride]));
    if (c - r < 0 && c + r >= lim) break;
  }
  dout[i] = (uint8_t)best;
}

// Edge pieces per edge (the same FP64 steps as the device kernel): nf[e] pieces of
// length <= h_s / 4, slots off[e]..off[e+1] of the sort.
int edge_layout(std::string* err, const SceneObj* S, std::vector<int64_t>& off, std::vector<int32_t>& nf) {
  const int64_t n_edges = (int64_t)S->edge_label_h.size();
  const double hs = S->params.voxel_size / S->params.dv;
  off.assign(n_edges + 1, 0);
  nf.assign(n_edges, 1);
  for (int64_t e = 0; e < n_edges; ++e) {
    const double* E = &S->edges_h[12 * e];
    double dx = E[3] - E[0], dy = E[4] - E[1], dz = E[5] - E[2];
    double L = std::sqrt(dx * dx + dy * dy + dz * dz);
    double q = std::ceil(L / (hs / 4.0));
    if (q > 1e8) {
      *err = "edge too long";
      return NIMBUS_ERR_ARG;
    }
    nf[e] = std::max(1, (int)q);
    off[e + 1] = off[e] + nf[e];
  }
  return NIMBUS_OK;
}

// Grid constants of the sort key and its width for the scene's grid, labels and edges.
int grid_keys(std::string* err, const SceneObj* S, GridK* g, int* key_bits) {
  const int dv = S->params.dv;
  const int64_t n_edges = (int64_t)S->edge_label_h.size();
  const int64_t n_cells = (int64_t)S->dims[0] * S->dims[1] * S->dims[2];
  for (int a = 0; a < 3; ++a) {
    g->o[a] = (float)S->origin[a];
    g->gmax[a] = S->dims[a] * dv - 1;
  }
  g->hs = (float)(S->params.voxel_size / dv);
  g->dv = dv;
  g->nx = S->dims[0];
  g->ny = S->dims[1];
  g->sub_bits = std::max(1, bits_for((uint64_t)dv * dv * dv - 1));
  uint64_t max_id = std::max<uint64_t>(S->max_label, n_edges > 0 ? (uint64_t)(n_edges - 1) : 0);
  g->id_bits = std::max(1, bits_for(max_id));
  *key_bits = bits_for((uint64_t)n_cells) + g->sub_bits + 1 + g->id_bits;
  if (*key_bits > 64) {
    *err = "sort key exceeds 64 bits (labels or grid too large)";
    return NIMBUS_ERR_ARG;
  }
  return NIMBUS_OK;
}

// Build every derived table of a scene from its device cloud on a fixed grid.
int build_tables(Mem& mem, SceneObj* S, cudaStream_t st) {
  std::string* err = mem.err;
  Scratch sc(&mem, st);
  const int dv = S->params.dv;
  const int64_t n = S->n_points;
  const int64_t n_edges = (int64_t)S->edge_label_h.size();
  const int64_t n_cells = (int64_t)S->dims[0] * S->dims[1] * S->dims[2];
  if (n_cells >= (1ll << 32)) {
    *err = "voxel grid too large";
    return NIMBUS_ERR_ARG;
  }
  const double h = S->params.voxel_size, hs = h / dv;
  std::vector<int64_t> off;
  std::vector<int32_t> nf;
  NB_TRY(edge_layout(err, S, off, nf));
  const int64_t n_piece_slots = off[n_edges];
  const int64_t n_total = n + n_piece_slots;
  if (n_total >= (1ll << 32) - 2) {
    *err = "too many points";
    return NIMBUS_ERR_ARG;
  }
  GridK g;
  int key_bits = 0;
  NB_TRY(grid_keys(err, S, &g, &key_bits));
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt, *flags, *ids, *counter;
  int4* pieces;
  int64_t* d_off;
  int32_t* d_nf;
  double* d_edges = nullptr;
  uint32_t* d_elabel = nullptr;
  NB_TRY(sc.get(&keys, n_total));
  NB_TRY(sc.get(&keys_alt, n_total));
  NB_TRY(sc.get(&vals, n_total));
  NB_TRY(sc.get(&vals_alt, n_total));
  NB_TRY(sc.get(&flags, n_total));
  NB_TRY(sc.get(&ids, n_total));
  NB_TRY(sc.get(&counter, 4));
  NB_TRY(sc.get(&pieces, std::max<int64_t>(1, n_piece_slots)));
  NB_TRY(sc.get(&d_off, n_edges + 1));
  NB_TRY(sc.get(&d_nf, std::max<int64_t>(1, n_edges)));
  NB_CUDA(err, cudaMemsetAsync(counter, 0, 4 * sizeof(uint32_t), st));
  const int B = 256;
  const unsigned G = std::min<unsigned>(grid_for(std::max<int64_t>(n_total, 1), B), 148u * 16u);
  if (n > 0) {
    k_point_keys<<<std::min<unsigned>(grid_for(n, B), 148u * 16u), B, 0, st>>>(g, S->xyz, S->label, n, keys, vals);
    NB_LAUNCHED(err);
  }
  if (n_edges > 0) {
    // edges live in the object's owned buffer (d.edges)
    d_edges = const_cast<double*>(S->d.edges);
    NB_TRY(sc.get(&d_elabel, n_edges));
    NB_CUDA(err, cudaMemcpyAsync(d_elabel, S->edge_label_h.data(), n_edges * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_off, off.data(), (n_edges + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_nf, nf.data(), n_edges * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    k_edge_pieces<<<grid_for(n_edges, 64), 64, 0, st>>>(g, d_edges, (int)n_edges, d_off, d_nf, n, keys, vals, pieces,
                                                         counter);
    NB_LAUNCHED(err);
  }
  NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, n_total, key_bits));
  k_run_flags<<<G, B, 0, st>>>(keys, n_total, flags);
  NB_LAUNCHED(err);
  NB_TRY(exclusive_scan(sc, flags, ids, n_total, counter + 1));
  uint32_t hc[2];
  NB_CUDA(err, cudaMemcpyAsync(hc, counter, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t n_valid = n + hc[0];
  const int64_t n_ie = hc[1];
  // owned tables: freed first if this is a rebuild
  for (void* p : S->table_bufs) mem.release(p, st);
  S->table_bufs.clear();
  auto own = [&](auto** p, size_t cnt) {
    int rc = mem.alloc_n(p, cnt, st);
    if (rc == NIMBUS_OK) S->table_bufs.push_back(*p);
    return rc;
  };
  // each IE's first entry and its voxel are kept for region updates
  uint32_t* starts;
  uint32_t* ie_cell;
  NB_TRY(own(&starts, n_ie + 1));
  NB_TRY(own(&ie_cell, std::max<int64_t>(1, n_ie)));
  k_run_starts<<<G, B, 0, st>>>(flags, ids, n_total, starts, (uint32_t)n_ie, (uint32_t)n_valid);
  NB_LAUNCHED(err);
  float4 *pts, *pnrm;
  IERec* ies;
  uint2* cells;
  uint8_t *march, *d1, *d2;
  NB_TRY(own(&pts, std::max<int64_t>(1, n_valid)));
  NB_TRY(own(&pnrm, std::max<int64_t>(1, n_valid)));
  NB_TRY(own(&ies, std::max<int64_t>(1, n_ie)));
  NB_TRY(own(&cells, n_cells));
  NB_TRY(own(&march, n_cells));
  NB_TRY(sc.get(&d1, n_cells));
  NB_TRY(sc.get(&d2, n_cells));
  if (n_valid > 0) {
    k_gather<<<std::min<unsigned>(grid_for(n_valid, B), 148u * 16u), B, 0, st>>>(vals, n_valid, n, S->xyz, S->nrm,
                                                                                  pts, pnrm);
    NB_LAUNCHED(err);
  }
  NB_CUDA(err, cudaMemsetAsync(cells, 0, n_cells * sizeof(uint2), st));
  if (n_ie > 0) {
    BuildK bk;
    bk.g = g;
    for (int a = 0; a < 3; ++a) bk.o[a] = S->origin[a];
    bk.hs = hs;
    bk.n_points = n;
    bk.n_ie = (int)n_ie;
    k_ie_build<<<grid_for(n_ie, 128), 128, 0, st>>>(bk, keys, vals, starts, pts, pnrm, S->material, pieces, d_edges,
                                                    ies, ie_cell);
    NB_LAUNCHED(err);
    if (n_edges > 0) {
      k_edge_labels<<<grid_for(n_ie, 256), 256, 0, st>>>(ies, (int)n_ie, d_elabel);
      NB_LAUNCHED(err);
    }
    k_cell_begin<<<grid_for(n_ie, 256), 256, 0, st>>>(ie_cell, (int)n_ie, cells);
    NB_LAUNCHED(err);
    k_cell_count<<<grid_for(n_ie, 256), 256, 0, st>>>(ie_cell, (int)n_ie, cells);
    NB_LAUNCHED(err);
  }
  const int nx = S->dims[0], ny = S->dims[1], nz = S->dims[2];
  k_march_x<<<grid_for((int64_t)ny * nz, 128), 128, 0, st>>>(cells, nx, ny, nz, d1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d1, d2, nx, ny, nz, 1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d2, march, nx, ny, nz, 2);
  NB_LAUNCHED(err);
  // the scratch buffers are released when sc leaves scope (stream-ordered)
  S->n_ie = n_ie;
  S->n_slots = n_valid;
  S->ie_start = starts;
  S->ie_cell = ie_cell;
  DScene& d = S->d;
  d.cells = cells;
  d.march = march;
  d.ies = ies;
  d.pts = pts;
  d.pnrm = pnrm;
  d.n_ie = (int)n_ie;
  return NIMBUS_OK;
}

void fill_dscene(SceneObj* S) {
  const nimbus_vox_params& p = S->params;
  DScene& d = S->d;
  double h = p.voxel_size, hs = h / p.dv;
  d.ox = (float)S->origin[0];
  d.oy = (float)S->origin[1];
  d.oz = (float)S->origin[2];
  d.h = (float)h;
  d.inv_h = (float)(1.0 / h);
  d.hs = (float)hs;
  d.inv_hs = (float)(1.0 / hs);
  d.nx = S->dims[0];
  d.ny = S->dims[1];
  d.nz = S->dims[2];
  d.dv = p.dv;
  d.odx = S->origin[0];
  d.ody = S->origin[1];
  d.odz = S->origin[2];
  d.hd = h;
  d.hsd = hs;
  d.n_cells = (long long)S->dims[0] * S->dims[1] * S->dims[2];
  d.n_edges = (int)S->edge_label_h.size();
  d.r_vox = (float)(h * std::sqrt(3.0) / 2.0);
  d.r_sub = (float)(hs * std::sqrt(3.0) / 2.0);
  d.seg_len = (float)(hs * std::sqrt(3.0));
  d.sdf_inv_s2 = (float)(1.0 / (p.sdf_sigma * p.sdf_sigma));
  d.sdf_eps = (float)p.sdf_eps;
  d.vis_ignore = (float)p.vis_ignore;
  d.sdf_max_steps = p.sdf_max_steps;
}

}  // namespace

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int copy_in(std::string* err, void* dst, const void* src, size_t n, cudaStream_t st) {
  if (n == 0) return NIMBUS_OK;
  NB_CUDA(err, cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, st));
  return NIMBUS_OK;
}

int voxelize_scene(Mem& mem, const nimbus_cloud* cloud, const nimbus_edges* edges, const nimbus_vox_params* p,
                   SceneObj* S, cudaStream_t st) {
  std::string* err = mem.err;
  if (!cloud || !p || cloud->n < 0 || (cloud->n > 0 && (!cloud->xyz || !cloud->nrm || !cloud->label))) {
    *err = "voxelize: invalid cloud";
    return NIMBUS_ERR_ARG;
  }
  if (!(p->voxel_size > 0) || p->dv < 1 || p->dv > 4 || p->sdf_max_steps < 1 || !(p->sdf_sigma > 0)) {
    *err = "voxelize: invalid parameters";
    return NIMBUS_ERR_ARG;
  }
  const int64_t n = cloud->n;
  const int64_t ne = edges ? edges->n : 0;
  if (ne < 0 || (ne > 0 && (!edges->edges || !edges->label))) {
    *err = "voxelize: invalid edges";
    return NIMBUS_ERR_ARG;
  }
  if (n == 0 && ne == 0 && !p->has_region) {
    *err = "voxelize: empty scene and no region";
    return NIMBUS_ERR_ARG;
  }
  S->mem = &mem;
  S->params = *p;
  S->n_points = n;
  NB_TRY(S->own(&S->xyz, std::max<int64_t>(1, 3 * n), st));
  NB_TRY(S->own(&S->nrm, std::max<int64_t>(1, 3 * n), st));
  NB_TRY(S->own(&S->label, std::max<int64_t>(1, n), st));
  NB_TRY(copy_in(err, S->xyz, cloud->xyz, 3 * n * sizeof(float), st));
  NB_TRY(copy_in(err, S->nrm, cloud->nrm, 3 * n * sizeof(float), st));
  NB_TRY(copy_in(err, S->label, cloud->label, n * sizeof(uint32_t), st));
  if (cloud->material) {
    NB_TRY(S->own(&S->material, std::max<int64_t>(1, n), st));
    NB_TRY(copy_in(err, S->material, cloud->material, n * sizeof(uint8_t), st));
  }
  S->edges_h.resize(12 * ne);
  S->edge_label_h.resize(ne);
  if (ne > 0) {
    NB_CUDA(err, cudaMemcpy(S->edges_h.data(), edges->edges, 12 * ne * sizeof(double), cudaMemcpyDefault));
    NB_CUDA(err, cudaMemcpy(S->edge_label_h.data(), edges->label, ne * sizeof(uint32_t), cudaMemcpyDefault));
    double* de;
    NB_TRY(S->own(&de, 12 * ne, st));
    NB_CUDA(err, cudaMemcpyAsync(de, S->edges_h.data(), 12 * ne * sizeof(double), cudaMemcpyHostToDevice, st));
    S->d.edges = de;
  }
  // bounds of the points (device reduction), the edges and the region (host)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  uint32_t maxlab = 0;
  if (n > 0) {
    uint32_t* red;
    Scratch sc(&mem, st);
    NB_TRY(sc.get(&red, 8));
    uint32_t init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
    NB_CUDA(err, cudaMemcpyAsync(red, init, sizeof init, cudaMemcpyHostToDevice, st));
    k_bounds<<<std::min<unsigned>(grid_for(n, 256), 148u * 8u), 256, 0, st>>>(S->xyz, S->label, n, red);
    NB_LAUNCHED(err);
    uint32_t hr[8];
    NB_CUDA(err, cudaMemcpyAsync(hr, red, sizeof hr, cudaMemcpyDeviceToHost, st));
    NB_CUDA(err, cudaStreamSynchronize(st));
    for (int a = 0; a < 6; ++a) {
      uint32_t u = hr[a];
      uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
      float f;
      std::memcpy(&f, &b, 4);
      if (a < 3) lo[a] = std::min(lo[a], (double)f);
      else hi[a - 3] = std::max(hi[a - 3], (double)f);
    }
    maxlab = hr[6];
  }
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], std::min(S->edges_h[12 * e + a], S->edges_h[12 * e + 3 + a]));
      hi[a] = std::max(hi[a], std::max(S->edges_h[12 * e + a], S->edges_h[12 * e + 3 + a]));
      maxlab = std::max(maxlab, S->edge_label_h[e]);
    }
  if (p->has_region)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p->region_min[a]);
      hi[a] = std::max(hi[a], p->region_max[a]);
    }
  if (maxlab >= (1u << 24)) {
    *err = "labels must be < 2^24";
    return NIMBUS_ERR_ARG;
  }
  S->max_label = maxlab;
  const double h = p->voxel_size;
  for (int a = 0; a < 3; ++a) {
    S->origin[a] = (std::floor(lo[a] / h) - 1.0) * h;
    double dd = std::ceil((hi[a] - S->origin[a]) / h) + 1.0;
    if (!(dd >= 1.0 && dd < 1e6)) {
      *err = "voxel grid dimensions out of range";
      return NIMBUS_ERR_ARG;
    }
    S->dims[a] = (int)dd;
  }
  fill_dscene(S);
  return build_tables(mem, S, st);
}

namespace {
__global__ void k_outside_flags(const float* __restrict__ xyz, int64_t n, float lx, float ly, float lz, float hx,
                                float hy, float hz, uint32_t* __restrict__ keep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    bool inside = x >= lx && x <= hx && y >= ly && y <= hy && z >= lz && z <= hz;
    keep[i] = inside ? 0u : 1u;
  }
}

__global__ void k_compact_points(const float* __restrict__ xyz, const float* __restrict__ nrm,
                                 const uint32_t* __restrict__ label, const uint8_t* __restrict__ mat, int64_t n,
                                 const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos,
                                 float* __restrict__ oxyz, float* __restrict__ onrm, uint32_t* __restrict__ olabel,
                                 uint8_t* __restrict__ omat) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    int64_t j = pos[i];
    for (int a = 0; a < 3; ++a) {
      oxyz[3 * j + a] = xyz[3 * i + a];
      onrm[3 * j + a] = nrm[3 * i + a];
    }
    olabel[j] = label[i];
    if (omat) omat[j] = mat ? mat[i] : 0;
  }
}
}  // namespace

// ----------------------------------------------------------- region-local rebuild
// A region update re-bins only the voxels whose points change: those that lose a
// point to the region or gain one from the replacement ("affected").  Their points
// and edge pieces are sorted on their own and reduced to IEs exactly as the full
// build does; the IEs and point entries of every other voxel are copied, in voxel
// order, to the positions a full build of the new cloud gives them.  The full
// build's order is a stable sort by (voxel, subvoxel, kind, label), so the result
// equals it entry for entry.
namespace {

__device__ __forceinline__ uint32_t cell_of_point(const GridK& g, const float* xyz) {
  int gs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gs[a] = subvoxel_axis(xyz[a], g.o[a], g.hs, g.gmax[a]);
  return (uint32_t)(((uint64_t)(gs[2] / g.dv) * g.ny + (gs[1] / g.dv)) * g.nx + (gs[0] / g.dv));
}

// Voxels of the points in [i0, i1) with want(i): marked affected.
__global__ void k_mark_cells(GridK g, const float* __restrict__ xyz, int64_t i0, int64_t i1,
                             const uint32_t* __restrict__ keep, uint32_t* __restrict__ aff) {
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x)
    if (!keep || !keep[i]) aff[cell_of_point(g, xyz + 3 * i)] = 1u;
}

__global__ void k_points_in_cells(GridK g, const float* __restrict__ xyz, int64_t n, const uint32_t* __restrict__ aff,
                                  uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = aff[cell_of_point(g, xyz + 3 * i)];
}

__global__ void k_edges_in_cells(const uint64_t* __restrict__ keys, int64_t n, int cell_shift,
                                 const uint32_t* __restrict__ aff, uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = keys[i] != INVALID_KEY && aff[keys[i] >> cell_shift] ? 1u : 0u;
}

// Local sort entries: the flagged points (new-cloud index as value), then the flagged
// edge-piece runs (value n_points + slot), each list in index order -- the order of
// equal keys in the full build's stable sort.
__global__ void k_local_entries(GridK g, const float* __restrict__ xyz, const uint32_t* __restrict__ label,
                                int64_t n_points, const uint32_t* __restrict__ pflag, const uint32_t* __restrict__ ppos,
                                const uint64_t* __restrict__ ekeys, int64_t n_slots, const uint32_t* __restrict__ eflag,
                                const uint32_t* __restrict__ epos, const uint32_t* __restrict__ m_pts,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t total = n_points + n_slots;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_points) {
      if (!pflag[i]) continue;
      int gs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) gs[a] = subvoxel_axis(xyz[3 * i + a], g.o[a], g.hs, g.gmax[a]);
      keys[ppos[i]] = pack_key(g, gs, IE_POINT, label[i]);
      vals[ppos[i]] = (uint32_t)i;
    } else {
      const int64_t e = i - n_points;
      if (!eflag[e]) continue;
      const uint32_t j = *m_pts + epos[e];
      keys[j] = ekeys[e];
      vals[j] = (uint32_t)(n_points + e);
    }
  }
}

// Per voxel: the local IE count, entry count and first local IE / entry.
__global__ void k_local_tally(const uint32_t* __restrict__ l_cell, const uint32_t* __restrict__ l_start, int64_t n_l,
                              uint32_t* __restrict__ cnt, uint32_t* __restrict__ ent, uint32_t* __restrict__ first_ie,
                              uint32_t* __restrict__ first_ent) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_l; j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = l_cell[j];
    atomicAdd(&cnt[c], 1u);
    atomicAdd(&ent[c], l_start[j + 1] - l_start[j]);
    if (j == 0 || l_cell[j - 1] != c) {
      first_ie[c] = (uint32_t)j;
      first_ent[c] = l_start[j];
    }
  }
}

// New IE and entry counts of every voxel: the local ones where affected, else the old.
__global__ void k_new_counts(const uint32_t* __restrict__ aff, const uint2* __restrict__ old_cells,
                             const uint32_t* __restrict__ old_start, const uint32_t* __restrict__ l_cnt,
                             const uint32_t* __restrict__ l_ent, int64_t n_cells, uint32_t* __restrict__ ie_cnt,
                             uint32_t* __restrict__ ent_cnt) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
    if (aff[c]) {
      ie_cnt[c] = l_cnt[c];
      ent_cnt[c] = l_ent[c];
    } else {
      const uint2 oc = old_cells[c];
      ie_cnt[c] = oc.y;
      ent_cnt[c] = oc.y ? old_start[oc.x + oc.y] - old_start[oc.x] : 0u;
    }
  }
}

__device__ __forceinline__ bool point_ie(const IERec& r) { return (__float_as_uint(r.nrm_meta.w) & 1u) == IE_POINT; }

// The IEs of unaffected voxels, moved to their new positions.
__global__ void k_splice_old_ies(const IERec* __restrict__ old_ies, const uint32_t* __restrict__ old_start,
                                 const uint32_t* __restrict__ old_cell, int64_t n_old, const uint2* __restrict__ old_cells,
                                 const uint32_t* __restrict__ aff, const uint32_t* __restrict__ ie_first,
                                 const uint32_t* __restrict__ ent_first, IERec* __restrict__ ies,
                                 uint32_t* __restrict__ starts, uint32_t* __restrict__ cellv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_old; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = old_cell[i];
    if (aff[c]) continue;
    const uint32_t c0 = old_cells[c].x;
    const uint32_t ni = ie_first[c] + ((uint32_t)i - c0), ne = ent_first[c] + (old_start[i] - old_start[c0]);
    IERec r = old_ies[i];
    if (point_ie(r)) r.bbc_pb.w = __uint_as_float(ne);
    ies[ni] = r;
    starts[ni] = ne;
    cellv[ni] = c;
  }
}

// Their point entries: moved, with each point's index in the cloud renumbered after
// the removal (new index = pos[old index]).
__global__ void k_splice_old_pts(const float4* __restrict__ old_pts, const float4* __restrict__ old_nrm, int64_t n_ent,
                                 const uint32_t* __restrict__ old_start, int64_t n_old, const uint32_t* __restrict__ old_cell,
                                 const IERec* __restrict__ old_ies, const uint2* __restrict__ old_cells,
                                 const uint32_t* __restrict__ aff, const uint32_t* __restrict__ ent_first,
                                 const uint32_t* __restrict__ pos, float4* __restrict__ pts, float4* __restrict__ nrm) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ent; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n_old;   // the IE of entry k: last i with old_start[i] <= k
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (old_start[mid] <= (uint32_t)k) lo = mid;
      else hi = mid;
    }
    const uint32_t c = old_cell[lo];
    if (aff[c]) continue;
    const uint32_t ne = ent_first[c] + ((uint32_t)k - old_start[old_cells[c].x]);
    float4 P = old_pts[k];
    if (point_ie(old_ies[lo])) P.w = __uint_as_float(pos[__float_as_uint(P.w)]);
    pts[ne] = P;
    nrm[ne] = old_nrm[k];
  }
}

// The rebuilt IEs of affected voxels and their entries, at their new positions.
__global__ void k_splice_new_ies(const IERec* __restrict__ l_ies, const uint32_t* __restrict__ l_start,
                                 const uint32_t* __restrict__ l_cell, int64_t n_l, const uint32_t* __restrict__ first_ie,
                                 const uint32_t* __restrict__ first_ent, const uint32_t* __restrict__ ie_first,
                                 const uint32_t* __restrict__ ent_first, IERec* __restrict__ ies,
                                 uint32_t* __restrict__ starts, uint32_t* __restrict__ cellv) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_l; j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = l_cell[j];
    const uint32_t ni = ie_first[c] + ((uint32_t)j - first_ie[c]), ne = ent_first[c] + (l_start[j] - first_ent[c]);
    IERec r = l_ies[j];
    if (point_ie(r)) r.bbc_pb.w = __uint_as_float(ne);
    ies[ni] = r;
    starts[ni] = ne;
    cellv[ni] = c;
  }
}

__global__ void k_splice_new_pts(const float4* __restrict__ l_pts, const float4* __restrict__ l_nrm, int64_t m,
                                 const uint32_t* __restrict__ l_flags, const uint32_t* __restrict__ l_ids,
                                 const uint32_t* __restrict__ l_cell, const uint32_t* __restrict__ first_ent,
                                 const uint32_t* __restrict__ ent_first, float4* __restrict__ pts,
                                 float4* __restrict__ nrm) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = l_ids[k] + l_flags[k] - 1u;   // local IE of entry k
    const uint32_t c = l_cell[j];
    const uint32_t ne = ent_first[c] + ((uint32_t)k - first_ent[c]);
    pts[ne] = l_pts[k];
    nrm[ne] = l_nrm[k];
  }
}

__global__ void k_new_cells(const uint32_t* __restrict__ ie_cnt, const uint32_t* __restrict__ ie_first, int64_t n_cells,
                            uint2* __restrict__ cells) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x)
    cells[c] = make_uint2(ie_cnt[c] ? ie_first[c] : 0u, ie_cnt[c]);
}

__global__ void k_set_last(uint32_t* __restrict__ starts, int64_t n_ie, const uint32_t* __restrict__ total) {
  starts[n_ie] = *total;
}

}  // namespace

// The tables of the scene's new cloud (already in S) from its old tables, given the
// affected voxels and the renumbering pos[] of the old cloud's kept points.
int splice_region(Mem& mem, SceneObj* S, const uint32_t* aff, const uint32_t* pos, cudaStream_t st) {
  std::string* err = mem.err;
  Scratch sc(&mem, st);
  const int64_t n = S->n_points, n_cells = (int64_t)S->dims[0] * S->dims[1] * S->dims[2];
  const int64_t n_edges = (int64_t)S->edge_label_h.size();
  const int64_t n_old = S->n_ie, n_old_ent = S->n_slots;
  std::vector<int64_t> off;
  std::vector<int32_t> nf;
  NB_TRY(edge_layout(err, S, off, nf));
  const int64_t n_slots = off[n_edges];
  GridK g;
  int key_bits = 0;
  NB_TRY(grid_keys(err, S, &g, &key_bits));
  const int cell_shift = g.sub_bits + 1 + g.id_bits;
  const int B = 256;
  auto grid = [&](int64_t m) { return std::min<unsigned>(grid_for(std::max<int64_t>(m, 1), B), 148u * 16u); };
  // entries of the affected voxels: points, then edge-piece runs
  uint32_t *pflag, *ppos, *cnt2;
  NB_TRY(sc.get(&pflag, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&ppos, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&cnt2, 4));
  NB_CUDA(err, cudaMemsetAsync(cnt2, 0, 4 * sizeof(uint32_t), st));
  if (n > 0) {
    k_points_in_cells<<<grid(n), B, 0, st>>>(g, S->xyz, n, aff, pflag);
    NB_LAUNCHED(err);
  }
  NB_TRY(exclusive_scan(sc, pflag, ppos, n, cnt2));
  uint64_t *ekeys = nullptr;
  uint32_t *evals = nullptr, *eflag = nullptr, *epos = nullptr, *d_elabel = nullptr;
  int4* pieces = nullptr;
  int64_t* d_off = nullptr;
  int32_t* d_nf = nullptr;
  NB_TRY(sc.get(&pieces, std::max<int64_t>(1, n_slots)));
  if (n_edges > 0) {
    NB_TRY(sc.get(&ekeys, n_slots));
    NB_TRY(sc.get(&evals, n_slots));
    NB_TRY(sc.get(&eflag, n_slots));
    NB_TRY(sc.get(&epos, n_slots));
    NB_TRY(sc.get(&d_off, n_edges + 1));
    NB_TRY(sc.get(&d_nf, n_edges));
    NB_TRY(sc.get(&d_elabel, n_edges));
    NB_CUDA(err, cudaMemcpyAsync(d_off, off.data(), (n_edges + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_nf, nf.data(), n_edges * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_elabel, S->edge_label_h.data(), n_edges * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, st));
    k_edge_pieces<<<grid_for(n_edges, 64), 64, 0, st>>>(g, S->d.edges, (int)n_edges, d_off, d_nf, 0, ekeys, evals,
                                                         pieces, cnt2 + 2);
    NB_LAUNCHED(err);
    k_edges_in_cells<<<grid(n_slots), B, 0, st>>>(ekeys, n_slots, cell_shift, aff, eflag);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(sc, eflag, epos, n_slots, cnt2 + 1));
  }
  uint32_t hm[2] = {0, 0};
  NB_CUDA(err, cudaMemcpyAsync(hm, cnt2, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t m = (int64_t)hm[0] + hm[1];
  // local sort and IE build (as in build_tables, on the affected voxels only)
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt, *flags, *ids, *l_n;
  NB_TRY(sc.get(&keys, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&keys_alt, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&vals, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&vals_alt, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&flags, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&ids, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&l_n, 1));
  if (m > 0) {
    k_local_entries<<<grid(n + n_slots), B, 0, st>>>(g, S->xyz, S->label, n, pflag, ppos, ekeys, n_edges > 0 ? n_slots : 0,
                                                    eflag, epos, cnt2, keys, vals);
    NB_LAUNCHED(err);
    NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, m, key_bits));
    k_run_flags<<<grid(m), B, 0, st>>>(keys, m, flags);
    NB_LAUNCHED(err);
  }
  NB_TRY(exclusive_scan(sc, flags, ids, m, l_n));
  uint32_t hl = 0;
  NB_CUDA(err, cudaMemcpyAsync(&hl, l_n, sizeof hl, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t n_l = hl;
  uint32_t *l_start, *l_cell;
  float4 *l_pts, *l_nrm;
  IERec* l_ies;
  NB_TRY(sc.get(&l_start, n_l + 1));
  NB_TRY(sc.get(&l_cell, std::max<int64_t>(1, n_l)));
  NB_TRY(sc.get(&l_pts, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&l_nrm, std::max<int64_t>(1, m)));
  NB_TRY(sc.get(&l_ies, std::max<int64_t>(1, n_l)));
  k_run_starts<<<grid(m), B, 0, st>>>(flags, ids, m, l_start, (uint32_t)n_l, (uint32_t)m);
  NB_LAUNCHED(err);
  if (m > 0) {
    k_gather<<<grid(m), B, 0, st>>>(vals, m, n, S->xyz, S->nrm, l_pts, l_nrm);
    NB_LAUNCHED(err);
  }
  if (n_l > 0) {
    BuildK bk;
    bk.g = g;
    for (int a = 0; a < 3; ++a) bk.o[a] = S->origin[a];
    bk.hs = S->params.voxel_size / S->params.dv;
    bk.n_points = n;
    bk.n_ie = (int)n_l;
    k_ie_build<<<grid_for(n_l, 128), 128, 0, st>>>(bk, keys, vals, l_start, l_pts, l_nrm, S->material, pieces,
                                                   S->d.edges, l_ies, l_cell);
    NB_LAUNCHED(err);
    if (n_edges > 0) {
      k_edge_labels<<<grid_for(n_l, 256), 256, 0, st>>>(l_ies, (int)n_l, d_elabel);
      NB_LAUNCHED(err);
    }
  }
  // new counts per voxel, and where each voxel's IEs and entries start
  uint32_t *l_cnt, *l_ent, *first_ie, *first_ent, *ie_cnt, *ent_cnt, *ie_first, *ent_first, *tot;
  NB_TRY(sc.get(&l_cnt, n_cells));
  NB_TRY(sc.get(&l_ent, n_cells));
  NB_TRY(sc.get(&first_ie, n_cells));
  NB_TRY(sc.get(&first_ent, n_cells));
  NB_TRY(sc.get(&ie_cnt, n_cells));
  NB_TRY(sc.get(&ent_cnt, n_cells));
  NB_TRY(sc.get(&ie_first, n_cells));
  NB_TRY(sc.get(&ent_first, n_cells));
  NB_TRY(sc.get(&tot, 2));
  NB_CUDA(err, cudaMemsetAsync(l_cnt, 0, n_cells * sizeof(uint32_t), st));
  NB_CUDA(err, cudaMemsetAsync(l_ent, 0, n_cells * sizeof(uint32_t), st));
  if (n_l > 0) {
    k_local_tally<<<grid(n_l), B, 0, st>>>(l_cell, l_start, n_l, l_cnt, l_ent, first_ie, first_ent);
    NB_LAUNCHED(err);
  }
  k_new_counts<<<grid(n_cells), B, 0, st>>>(aff, S->d.cells, S->ie_start, l_cnt, l_ent, n_cells, ie_cnt, ent_cnt);
  NB_LAUNCHED(err);
  NB_TRY(exclusive_scan(sc, ie_cnt, ie_first, n_cells, tot));
  NB_TRY(exclusive_scan(sc, ent_cnt, ent_first, n_cells, tot + 1));
  uint32_t ht[2] = {0, 0};
  NB_CUDA(err, cudaMemcpyAsync(ht, tot, sizeof ht, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t n_ie = ht[0], n_valid = ht[1];
  // the new tables
  std::vector<void*> old_bufs = S->table_bufs;
  std::vector<void*> bufs;
  auto own = [&](auto** p, size_t c) {
    int rc = mem.alloc_n(p, c, st);
    if (rc == NIMBUS_OK) bufs.push_back(*p);
    return rc;
  };
  auto drop_new = [&]() {
    for (void* p : bufs) mem.release(p, st);
  };
  uint32_t *starts, *cellv;
  float4 *pts, *pnrm;
  IERec* ies;
  uint2* cells;
  uint8_t *march, *d1, *d2;
  int rc = NIMBUS_OK;
  if ((rc = own(&starts, n_ie + 1)) != NIMBUS_OK || (rc = own(&cellv, std::max<int64_t>(1, n_ie))) != NIMBUS_OK ||
      (rc = own(&pts, std::max<int64_t>(1, n_valid))) != NIMBUS_OK ||
      (rc = own(&pnrm, std::max<int64_t>(1, n_valid))) != NIMBUS_OK ||
      (rc = own(&ies, std::max<int64_t>(1, n_ie))) != NIMBUS_OK || (rc = own(&cells, n_cells)) != NIMBUS_OK ||
      (rc = own(&march, n_cells)) != NIMBUS_OK) {
    drop_new();
    return rc;
  }
  NB_TRY(sc.get(&d1, n_cells));
  NB_TRY(sc.get(&d2, n_cells));
  if (n_old > 0) {
    k_splice_old_ies<<<grid(n_old), B, 0, st>>>(S->d.ies, S->ie_start, S->ie_cell, n_old, S->d.cells, aff, ie_first,
                                               ent_first, ies, starts, cellv);
    NB_LAUNCHED(err);
  }
  if (n_old_ent > 0) {
    k_splice_old_pts<<<grid(n_old_ent), B, 0, st>>>(S->d.pts, S->d.pnrm, n_old_ent, S->ie_start, n_old, S->ie_cell,
                                                   S->d.ies, S->d.cells, aff, ent_first, pos, pts, pnrm);
    NB_LAUNCHED(err);
  }
  if (n_l > 0) {
    k_splice_new_ies<<<grid(n_l), B, 0, st>>>(l_ies, l_start, l_cell, n_l, first_ie, first_ent, ie_first, ent_first, ies,
                                             starts, cellv);
    NB_LAUNCHED(err);
    k_splice_new_pts<<<grid(m), B, 0, st>>>(l_pts, l_nrm, m, flags, ids, l_cell, first_ent, ent_first, pts, pnrm);
    NB_LAUNCHED(err);
  }
  k_set_last<<<1, 1, 0, st>>>(starts, n_ie, tot + 1);
  NB_LAUNCHED(err);
  k_new_cells<<<grid(n_cells), B, 0, st>>>(ie_cnt, ie_first, n_cells, cells);
  NB_LAUNCHED(err);
  const int nx = S->dims[0], ny = S->dims[1], nz = S->dims[2];
  k_march_x<<<grid_for((int64_t)ny * nz, 128), 128, 0, st>>>(cells, nx, ny, nz, d1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d1, d2, nx, ny, nz, 1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d2, march, nx, ny, nz, 2);
  NB_LAUNCHED(err);
  // swap the tables (the old ones are released stream-ordered after the copies)
  for (void* p : old_bufs) mem.release(p, st);
  S->table_bufs = bufs;
  S->n_ie = n_ie;
  S->n_slots = n_valid;
  S->ie_start = starts;
  S->ie_cell = cellv;
  DScene& d = S->d;
  d.cells = cells;
  d.march = march;
  d.ies = ies;
  d.pts = pts;
  d.pnrm = pnrm;
  d.n_ie = (int)n_ie;
  return NIMBUS_OK;
}

int update_scene_region(Mem& mem, SceneObj* S, const double lo[3], const double hi[3], const nimbus_cloud* repl,
                        cudaStream_t st) {
  std::string* err = mem.err;
  const int64_t n = S->n_points;
  const int64_t nr = repl ? repl->n : 0;
  if (nr < 0 || (nr > 0 && (!repl->xyz || !repl->nrm || !repl->label))) {
    *err = "update_region: invalid replacement cloud";
    return NIMBUS_ERR_ARG;
  }
  Scratch sc(&mem, st);
  uint32_t *keep, *pos, *cnt;
  NB_TRY(sc.get(&keep, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&pos, std::max<int64_t>(1, n)));
  NB_TRY(sc.get(&cnt, 1));
  if (n > 0) {
    k_outside_flags<<<std::min<unsigned>(grid_for(n, 256), 148u * 8u), 256, 0, st>>>(
        S->xyz, n, (float)lo[0], (float)lo[1], (float)lo[2], (float)hi[0], (float)hi[1], (float)hi[2], keep);
    NB_LAUNCHED(err);
  }
  NB_TRY(exclusive_scan(sc, keep, pos, n, cnt));
  // voxels that lose points (marked now, on the old cloud) or gain replacement
  // points (marked below) are the only ones re-binned
  const int64_t n_cells = (int64_t)S->dims[0] * S->dims[1] * S->dims[2];
  const bool local = S->ie_start != nullptr && S->ie_cell != nullptr;
  uint32_t* aff = nullptr;
  GridK gm;
  int kb_unused = 0;
  if (local) {
    NB_TRY(grid_keys(err, S, &gm, &kb_unused));
    NB_TRY(sc.get(&aff, n_cells));
    NB_CUDA(err, cudaMemsetAsync(aff, 0, n_cells * sizeof(uint32_t), st));
    if (n > 0) {
      k_mark_cells<<<std::min<unsigned>(grid_for(n, 256), 148u * 8u), 256, 0, st>>>(gm, S->xyz, 0, n, keep, aff);
      NB_LAUNCHED(err);
    }
  }
  uint32_t n_keep = 0;
  NB_CUDA(err, cudaMemcpyAsync(&n_keep, cnt, sizeof n_keep, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t n_new = (int64_t)n_keep + nr;
  float *nxyz, *nnrm;
  uint32_t* nlab;
  uint8_t* nmat = nullptr;
  NB_TRY(mem.alloc_n(&nxyz, std::max<int64_t>(1, 3 * n_new), st));
  NB_TRY(mem.alloc_n(&nnrm, std::max<int64_t>(1, 3 * n_new), st));
  NB_TRY(mem.alloc_n(&nlab, std::max<int64_t>(1, n_new), st));
  bool with_mat = S->material != nullptr || (repl && repl->material);
  if (with_mat) NB_TRY(mem.alloc_n(&nmat, std::max<int64_t>(1, n_new), st));
  if (n > 0) {
    k_compact_points<<<std::min<unsigned>(grid_for(n, 256), 148u * 8u), 256, 0, st>>>(
        S->xyz, S->nrm, S->label, S->material, n, keep, pos, nxyz, nnrm, nlab, nmat);
    NB_LAUNCHED(err);
  }
  if (nr > 0) {
    NB_TRY(copy_in(err, nxyz + 3 * n_keep, repl->xyz, 3 * nr * sizeof(float), st));
    NB_TRY(copy_in(err, nnrm + 3 * n_keep, repl->nrm, 3 * nr * sizeof(float), st));
    NB_TRY(copy_in(err, nlab + n_keep, repl->label, nr * sizeof(uint32_t), st));
    if (nmat) {
      if (repl->material) NB_TRY(copy_in(err, nmat + n_keep, repl->material, nr, st));
      else NB_CUDA(err, cudaMemsetAsync(nmat + n_keep, 0, nr, st));
    }
    // the replacement must lie on the existing grid and keep labels < 2^24
    std::vector<uint32_t> hl(nr);
    NB_CUDA(err, cudaMemcpy(hl.data(), repl->label, nr * sizeof(uint32_t), cudaMemcpyDefault));
    for (uint32_t l : hl) S->max_label = std::max(S->max_label, l);
  }
  // swap in the new cloud
  auto swap_buf = [&](void* oldp, void* newp) {
    for (auto& b : S->bufs)
      if (b == oldp) b = newp;
    mem.release(oldp, st);
  };
  swap_buf(S->xyz, nxyz);
  swap_buf(S->nrm, nnrm);
  swap_buf(S->label, nlab);
  if (S->material) swap_buf(S->material, nmat);
  else if (nmat) S->bufs.push_back(nmat);
  S->xyz = nxyz;
  S->nrm = nnrm;
  S->label = nlab;
  S->material = nmat;
  S->n_points = n_new;
  if (!local) return build_tables(mem, S, st);
  if (nr > 0) {
    k_mark_cells<<<std::min<unsigned>(grid_for(nr, 256), 148u * 8u), 256, 0, st>>>(gm, nxyz, n_keep, n_new, nullptr,
                                                                                   aff);
    NB_LAUNCHED(err);
  }
  return splice_region(mem, S, aff, pos, st);
}

// ----------------------------------------------------------- scene checkpoint
namespace {
constexpr char kMagic[8] = {'N', 'I', 'M', 'B', 'U', 'S', 'C', '1'};
constexpr uint32_t kVersion = 1;

struct Fnv {   // FNV-1a over the payload
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  }
};

struct Writer {
  FILE* f;
  Fnv sum;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (n == 0) return;
    sum.add(p, n);
    ok = ok && std::fwrite(p, 1, n, f) == n;
  }
};

struct Reader {
  FILE* f;
  Fnv sum;
  bool ok = true;
  void get(void* p, size_t n) {
    if (n == 0 || !ok) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) sum.add(p, n);
  }
};
}  // namespace

int scene_save(Mem& mem, SceneObj* S, const char* path, cudaStream_t st) {
  std::string* err = mem.err;
  if (!path) {
    *err = "scene_save: null path";
    return NIMBUS_ERR_ARG;
  }
  const int64_t n = S->n_points, ne = (int64_t)S->edge_label_h.size();
  std::vector<float> xyz(3 * n), nrm(3 * n);
  std::vector<uint32_t> lab(n);
  std::vector<uint8_t> mat(S->material ? n : 0);
  NB_CUDA(err, cudaStreamSynchronize(st));
  if (n > 0) {
    NB_CUDA(err, cudaMemcpy(xyz.data(), S->xyz, xyz.size() * sizeof(float), cudaMemcpyDeviceToHost));
    NB_CUDA(err, cudaMemcpy(nrm.data(), S->nrm, nrm.size() * sizeof(float), cudaMemcpyDeviceToHost));
    NB_CUDA(err, cudaMemcpy(lab.data(), S->label, lab.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (S->material) NB_CUDA(err, cudaMemcpy(mat.data(), S->material, mat.size(), cudaMemcpyDeviceToHost));
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    *err = std::string("scene_save: cannot open ") + path;
    return NIMBUS_ERR_IO;
  }
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
  Writer w{f};
  const uint32_t has_mat = S->material ? 1u : 0u;
  w.put(&kVersion, 4);
  w.put(&S->params, sizeof S->params);
  w.put(S->origin, sizeof S->origin);
  w.put(S->dims, sizeof S->dims);
  w.put(&n, 8);
  w.put(&ne, 8);
  w.put(&S->max_label, 4);
  w.put(&has_mat, 4);
  w.put(xyz.data(), xyz.size() * sizeof(float));
  w.put(nrm.data(), nrm.size() * sizeof(float));
  w.put(lab.data(), lab.size() * sizeof(uint32_t));
  w.put(mat.data(), mat.size());
  w.put(S->edges_h.data(), S->edges_h.size() * sizeof(double));
  w.put(S->edge_label_h.data(), S->edge_label_h.size() * sizeof(uint32_t));
  ok = ok && w.ok && std::fwrite(&w.sum.h, 1, 8, f) == 8;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    *err = std::string("scene_save: write failed: ") + path;
    return NIMBUS_ERR_IO;
  }
  return NIMBUS_OK;
}

int scene_load(Mem& mem, const char* path, SceneObj* S, cudaStream_t st) {
  std::string* err = mem.err;
  if (!path) {
    *err = "scene_load: null path";
    return NIMBUS_ERR_ARG;
  }
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    *err = std::string("scene_load: cannot open ") + path;
    return NIMBUS_ERR_IO;
  }
  auto fail = [&](const char* why) {
    std::fclose(f);
    *err = std::string("scene_load: ") + why + ": " + path;
    return NIMBUS_ERR_IO;
  };
  char magic[8];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0) return fail("not a scene checkpoint");
  Reader r{f};
  uint32_t version = 0, has_mat = 0;
  int64_t n = 0, ne = 0;
  r.get(&version, 4);
  if (!r.ok || version != kVersion) return fail("unsupported checkpoint version");
  r.get(&S->params, sizeof S->params);
  r.get(S->origin, sizeof S->origin);
  r.get(S->dims, sizeof S->dims);
  r.get(&n, 8);
  r.get(&ne, 8);
  r.get(&S->max_label, 4);
  r.get(&has_mat, 4);
  if (!r.ok || n < 0 || n > (int64_t)1 << 36 || ne < 0 || ne > (int64_t)1 << 28 || has_mat > 1 ||
      !(S->params.voxel_size > 0) || S->params.dv < 1 || S->params.dv > 4 || S->max_label >= (1u << 24))
    return fail("damaged header");
  for (int a = 0; a < 3; ++a)
    if (S->dims[a] < 1 || S->dims[a] >= 1000000) return fail("damaged header");
  std::vector<float> xyz(3 * n), nrm(3 * n);
  std::vector<uint32_t> lab(n);
  std::vector<uint8_t> mat(has_mat ? n : 0);
  S->edges_h.resize(12 * ne);
  S->edge_label_h.resize(ne);
  r.get(xyz.data(), xyz.size() * sizeof(float));
  r.get(nrm.data(), nrm.size() * sizeof(float));
  r.get(lab.data(), lab.size() * sizeof(uint32_t));
  r.get(mat.data(), mat.size());
  r.get(S->edges_h.data(), S->edges_h.size() * sizeof(double));
  r.get(S->edge_label_h.data(), S->edge_label_h.size() * sizeof(uint32_t));
  uint64_t sum = 0;
  const bool got_sum = r.ok && std::fread(&sum, 1, 8, f) == 8;
  if (!got_sum) return fail("truncated checkpoint");
  if (sum != r.sum.h) return fail("checksum mismatch");
  std::fclose(f);
  S->mem = &mem;
  S->n_points = n;
  NB_TRY(S->own(&S->xyz, std::max<int64_t>(1, 3 * n), st));
  NB_TRY(S->own(&S->nrm, std::max<int64_t>(1, 3 * n), st));
  NB_TRY(S->own(&S->label, std::max<int64_t>(1, n), st));
  if (n > 0) {
    NB_CUDA(err, cudaMemcpyAsync(S->xyz, xyz.data(), xyz.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(S->nrm, nrm.data(), nrm.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(S->label, lab.data(), lab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  }
  if (has_mat) {
    NB_TRY(S->own(&S->material, std::max<int64_t>(1, n), st));
    if (n > 0) NB_CUDA(err, cudaMemcpyAsync(S->material, mat.data(), mat.size(), cudaMemcpyHostToDevice, st));
  }
  if (ne > 0) {
    double* de;
    NB_TRY(S->own(&de, 12 * ne, st));
    NB_CUDA(err, cudaMemcpyAsync(de, S->edges_h.data(), 12 * ne * sizeof(double), cudaMemcpyHostToDevice, st));
    S->d.edges = de;
  }
  fill_dscene(S);
  const int rc = build_tables(mem, S, st);
  if (rc == NIMBUS_OK) NB_CUDA(err, cudaStreamSynchronize(st));   // the host vectors go out of scope
  return rc;
}

// ----------------------------------------------------------- voxelisation without allocation
// Every intermediate of nimbus_voxelize_static lives in this one fixed device array:
// 152.5 bytes per point (sort keys and values with their work copies, run flags and
// ids, run starts, grouped points, 80-byte entity records) plus 10 bytes per voxel and a
// small reserve for the scan and sort tables, for the largest sizes allowed.
namespace {
constexpr size_t kStaticPoints = NIMBUS_STATIC_MAX_POINTS;
constexpr size_t kStaticCells = NIMBUS_STATIC_MAX_CELLS;
constexpr size_t kStaticBytes = 153 * kStaticPoints + 10 * kStaticCells + (4u << 20);
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

// Device address of g_static_scratch on each device, resolved once per device with
// that device current (the host-side name is only a stand-in for the symbol).
std::mutex g_static_mu;
void* g_static_addr[128] = {nullptr};

int static_scratch(std::string* err, void** out) {
  int dev = 0;
  NB_CUDA(err, cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    *err = "device index out of range";
    return NIMBUS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    NB_CUDA(err, cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return NIMBUS_OK;
}

// Entity records and voxel ranges -> the caller's structure-of-arrays buffers.
__global__ void k_static_out(const IERec* __restrict__ ies, int n_ie, const uint2* __restrict__ cells,
                             int64_t n_cells, nimbus_static_tables o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ie; i += (int64_t)gridDim.x * blockDim.x) {
    const IERec r = ies[i];
    o.kind[i] = (int32_t)(__float_as_uint(r.nrm_meta.w) & 1u);
    o.label[i] = __float_as_uint(r.rp_lab.w);
    o.material[i] = (uint8_t)((__float_as_uint(r.nrm_meta.w) >> 8) & 0xffu);
    o.pcount[i] = (int32_t)__float_as_uint(r.sc_pc.w);
    const float rp[3] = {r.rp_lab.x, r.rp_lab.y, r.rp_lab.z};
    const float nn[3] = {r.nrm_meta.x, r.nrm_meta.y, r.nrm_meta.z};
    const float bb[3] = {r.bbc_pb.x, r.bbc_pb.y, r.bbc_pb.z};
    for (int a = 0; a < 3; ++a) {
      o.rp[3 * i + a] = rp[a];
      o.normal[3 * i + a] = nn[a];
      o.bbc[3 * i + a] = bb[a];
    }
  }
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
    o.cell_begin[c] = cells[c].y ? cells[c].x : 0u;
    o.cell_count[c] = cells[c].y;
  }
}

__global__ void k_static_gs(const IERec* __restrict__ ies, int n_ie, float ox, float oy, float oz, float hs,
                            int32_t* __restrict__ gs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ie) return;
  const float4 sc = ies[i].sc_pc;
  gs[3 * i] = (int32_t)floorf((sc.x - ox) / hs);
  gs[3 * i + 1] = (int32_t)floorf((sc.y - oy) / hs);
  gs[3 * i + 2] = (int32_t)floorf((sc.z - oz) / hs);
}

}  // namespace

int voxelize_static(std::string* err, const nimbus_cloud* cloud, const nimbus_vox_params* p,
                    const nimbus_static_tables* out, nimbus_static_info* info, cudaStream_t st) {
  if (!cloud || !p || !out || !info || cloud->n < 1 || !cloud->xyz || !cloud->nrm || !cloud->label) {
    *err = "voxelize_static: invalid arguments";
    return NIMBUS_ERR_ARG;
  }
  if (!(p->voxel_size > 0) || p->dv < 1 || p->dv > 4 || p->sdf_max_steps < 1 || !(p->sdf_sigma > 0)) {
    *err = "voxelize_static: invalid parameters";
    return NIMBUS_ERR_ARG;
  }
  const int64_t n = cloud->n;
  if (n > (int64_t)kStaticPoints) {
    *err = "voxelize_static: the cloud has more than NIMBUS_STATIC_MAX_POINTS points";
    return NIMBUS_ERR_ARG;
  }
  if (!is_device_ptr(cloud->xyz) || !is_device_ptr(cloud->nrm) || !is_device_ptr(cloud->label) ||
      (cloud->material && !is_device_ptr(cloud->material))) {
    *err = "voxelize_static: inputs must be device pointers";
    return NIMBUS_ERR_ARG;
  }
  // every output a non-zero capacity promises must be a device buffer: a null or
  // host pointer is refused here, before any device work writes through it
  if (out->ie_capacity < 0 || out->cell_capacity < 0) {
    *err = "voxelize_static: negative output capacity";
    return NIMBUS_ERR_ARG;
  }
  if (out->ie_capacity > 0) {
    const void* ie_out[8] = {out->kind, out->label, out->gs, out->pcount, out->rp, out->normal, out->bbc,
                             out->material};
    for (const void* q : ie_out)
      if (!q || !is_device_ptr(q)) {
        *err = "voxelize_static: entity outputs must be device pointers";
        return NIMBUS_ERR_ARG;
      }
  }
  if (out->cell_capacity > 0) {
    const void* cell_out[3] = {out->cell_begin, out->cell_count, out->march};
    for (const void* q : cell_out)
      if (!q || !is_device_ptr(q)) {
        *err = "voxelize_static: voxel outputs must be device pointers";
        return NIMBUS_ERR_ARG;
      }
  }
  void* base = nullptr;
  NB_TRY(static_scratch(err, &base));
  Mem m;  // error sink only: the arena below serves every buffer
  m.err = err;
  Scratch sc(&m, st);
  sc.arena = static_cast<char*>(base);
  sc.arena_cap = kStaticBytes;
  // bounds of the cloud (counters cleared first: the array keeps the last call's contents)
  uint32_t* red;
  NB_TRY(sc.get(&red, 8));
  NB_CUDA(err, cudaMemsetAsync(red, 0xff, 3 * sizeof(uint32_t), st));
  NB_CUDA(err, cudaMemsetAsync(red + 3, 0, 5 * sizeof(uint32_t), st));
  k_bounds<<<std::min<unsigned>(grid_for(n, 256), 148u * 8u), 256, 0, st>>>(cloud->xyz, cloud->label, n, red);
  NB_LAUNCHED(err);
  uint32_t hr[8];
  NB_CUDA(err, cudaMemcpyAsync(hr, red, sizeof hr, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  double lo[3], hi[3];
  for (int a = 0; a < 6; ++a) {
    uint32_t u = hr[a];
    uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    std::memcpy(&f, &b, 4);
    if (a < 3) lo[a] = (double)f;
    else hi[a - 3] = (double)f;
  }
  if (p->has_region)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p->region_min[a]);
      hi[a] = std::max(hi[a], p->region_max[a]);
    }
  const uint32_t maxlab = hr[6];
  if (maxlab >= (1u << 24)) {
    *err = "voxelize_static: labels must be < 2^24";
    return NIMBUS_ERR_ARG;
  }
  const double h = p->voxel_size, hs = h / p->dv;
  int dims[3];
  double origin[3];
  for (int a = 0; a < 3; ++a) {
    origin[a] = (std::floor(lo[a] / h) - 1.0) * h;
    double dd = std::ceil((hi[a] - origin[a]) / h) + 1.0;
    if (!(dd >= 1.0 && dd < 1e6)) {
      *err = "voxelize_static: voxel grid dimensions out of range";
      return NIMBUS_ERR_ARG;
    }
    dims[a] = (int)dd;
    info->origin[a] = origin[a];
    info->dims[a] = dims[a];
  }
  const int64_t n_cells = (int64_t)dims[0] * dims[1] * dims[2];
  info->n_cells = n_cells;
  info->n_ie = 0;
  if (n_cells > (int64_t)kStaticCells) {
    *err = "voxelize_static: the voxel grid has more than NIMBUS_STATIC_MAX_CELLS voxels";
    return NIMBUS_ERR_ARG;
  }
  if (n_cells > out->cell_capacity) {   // known before the sort: no work spent on it
    info->n_ie = -1;                     // not counted yet
    *err = "voxelize_static: output capacity too small (needed sizes in info)";
    return NIMBUS_ERR_OVERFLOW;
  }
  GridK g;
  for (int a = 0; a < 3; ++a) {
    g.o[a] = (float)origin[a];
    g.gmax[a] = dims[a] * p->dv - 1;
  }
  g.hs = (float)hs;
  g.dv = p->dv;
  g.nx = dims[0];
  g.ny = dims[1];
  g.sub_bits = std::max(1, bits_for((uint64_t)p->dv * p->dv * p->dv - 1));
  g.id_bits = std::max(1, bits_for(maxlab));
  const int key_bits = bits_for((uint64_t)n_cells) + g.sub_bits + 1 + g.id_bits;
  if (key_bits > 64) {
    *err = "voxelize_static: sort key exceeds 64 bits";
    return NIMBUS_ERR_ARG;
  }
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt, *flags, *ids, *counter;
  NB_TRY(sc.get(&keys, n));
  NB_TRY(sc.get(&keys_alt, n));
  NB_TRY(sc.get(&vals, n));
  NB_TRY(sc.get(&vals_alt, n));
  NB_TRY(sc.get(&flags, n));
  NB_TRY(sc.get(&ids, n));
  NB_TRY(sc.get(&counter, 4));
  NB_CUDA(err, cudaMemsetAsync(counter, 0, 4 * sizeof(uint32_t), st));
  const int B = 256;
  const unsigned G = std::min<unsigned>(grid_for(n, B), 148u * 16u);
  k_point_keys<<<G, B, 0, st>>>(g, cloud->xyz, cloud->label, n, keys, vals);
  NB_LAUNCHED(err);
  NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, n, key_bits));
  k_run_flags<<<G, B, 0, st>>>(keys, n, flags);
  NB_LAUNCHED(err);
  NB_TRY(exclusive_scan(sc, flags, ids, n, counter + 1));
  uint32_t hn = 0;
  NB_CUDA(err, cudaMemcpyAsync(&hn, counter + 1, sizeof hn, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaStreamSynchronize(st));
  const int64_t n_ie = hn;
  info->n_ie = n_ie;
  if (n_ie > out->ie_capacity || n_cells > out->cell_capacity) {
    *err = "voxelize_static: output capacity too small (needed sizes in info)";
    return NIMBUS_ERR_OVERFLOW;
  }
  uint32_t *starts, *ie_cell;
  float4 *pts, *pnrm;
  IERec* ies;
  uint2* cells;
  uint8_t *d1, *d2;
  NB_TRY(sc.get(&starts, n_ie + 1));
  NB_TRY(sc.get(&ie_cell, std::max<int64_t>(1, n_ie)));
  NB_TRY(sc.get(&pts, n));
  NB_TRY(sc.get(&pnrm, n));
  NB_TRY(sc.get(&ies, std::max<int64_t>(1, n_ie)));
  NB_TRY(sc.get(&cells, n_cells));
  NB_TRY(sc.get(&d1, n_cells));
  NB_TRY(sc.get(&d2, n_cells));
  k_run_starts<<<G, B, 0, st>>>(flags, ids, n, starts, (uint32_t)n_ie, (uint32_t)n);
  NB_LAUNCHED(err);
  k_gather<<<G, B, 0, st>>>(vals, n, n, cloud->xyz, cloud->nrm, pts, pnrm);
  NB_LAUNCHED(err);
  NB_CUDA(err, cudaMemsetAsync(cells, 0, n_cells * sizeof(uint2), st));
  BuildK bk;
  bk.g = g;
  for (int a = 0; a < 3; ++a) bk.o[a] = origin[a];
  bk.hs = hs;
  bk.n_points = n;
  bk.n_ie = (int)n_ie;
  k_ie_build<<<grid_for(n_ie, 128), 128, 0, st>>>(bk, keys, vals, starts, pts, pnrm, cloud->material, nullptr,
                                                  nullptr, ies, ie_cell);
  NB_LAUNCHED(err);
  k_cell_begin<<<grid_for(n_ie, 256), 256, 0, st>>>(ie_cell, (int)n_ie, cells);
  NB_LAUNCHED(err);
  k_cell_count<<<grid_for(n_ie, 256), 256, 0, st>>>(ie_cell, (int)n_ie, cells);
  NB_LAUNCHED(err);
  k_march_x<<<grid_for((int64_t)dims[1] * dims[2], 128), 128, 0, st>>>(cells, dims[0], dims[1], dims[2], d1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d1, d2, dims[0], dims[1], dims[2], 1);
  NB_LAUNCHED(err);
  k_march_axis<<<grid_for(n_cells, 256), 256, 0, st>>>(d2, out->march, dims[0], dims[1], dims[2], 2);
  NB_LAUNCHED(err);
  k_static_out<<<std::min<unsigned>(grid_for(std::max<int64_t>(n_ie, n_cells), 256), 148u * 16u), 256, 0, st>>>(
      ies, (int)n_ie, cells, n_cells, *out);
  NB_LAUNCHED(err);
  k_static_gs<<<grid_for(n_ie, 256), 256, 0, st>>>(ies, (int)n_ie, (float)origin[0], (float)origin[1],
                                                  (float)origin[2], (float)hs, out->gs);
  NB_LAUNCHED(err);
  NB_CUDA(err, cudaStreamSynchronize(st));
  return NIMBUS_OK;
}

}  // namespace nb
