// Coarse path tracing (Section 2.2): transmission phase, propagation phase and
// voxel cone tracing, followed by the kappa duplicate limit.
//
// B300 design.  Level-synchronous: one launch per interaction depth, each a
// grid-stride loop over cone tasks (a reflection node is one task, a diffraction
// node one task per Keller-fan ray), sized to the SM count and reading its task
// count from device memory, so the whole level sequence runs without host round
// trips.  Traversal and hit tests are FP32.  Children are appended to
// structure-of-arrays node buffers of the next level with one atomic per child.
// TX visibility of every IE is computed once per TX (the paper's transmission
// phase casts a ray toward each IE) and reused by the uniform launch's cones.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nimbus_host.hpp"
#include "warp_geom.cuh"

namespace nb {

namespace {

constexpr double PI_D = 3.14159265358979323846;
constexpr int MAX_LEVELS = NB_MAXI + 1;
constexpr uint32_t NO_NODE = 0xFFFFFFFFu;

enum { CONE_PRIMARY = 0, CONE_REFLECT = 1, CONE_DIFFRACT = 2 };
// per-stage counters: [stage * N_STATS + ST_*] for stages vis tables, primary, levels
enum { ST_CONES = 0, ST_VIS = 1, ST_BYTES = 2, ST_EVALS = 3, ST_NO_RX = 4, N_STATS = 5 };
enum { STAGE_VIS = 0, STAGE_PRIMARY = 1, STAGE_LEVELS = 2, N_STAGES = 3 };

struct DTrace {
  float sin_a, cos_a, sin_a0, cos_a0;
  int M;
  float dphi, sep_eps;
  int max_refl, max_diff, max_int;
  int n_launch, n_tx, n_rx;
  uint32_t n_ie, n_edges;    // the scene's IE and edge counts (self-checks)
  double golden;
  const float4* tx;          // xyz
  const float4* rx;          // xyz
  const uint8_t* march;      // scene march field with the RX voxels folded in
  const uint32_t* rx_bits;   // one bit per voxel: it holds an RX
  const uint64_t* rx_sorted; // (voxel << 32) | rx, ascending
  int n_rx_sorted;
  const uint32_t* vis_ie;    // [n_tx * ie_words] TX -> IE visibility bits
  int ie_words;
  const uint32_t* vis_rx;    // [n_tx * n_rx]
  const int32_t* rx_owner;   // [n_rx] TX allowed to reach each RX (-1: any), or null
  const int32_t* rx_max_int; // [n_rx] interaction limit of each RX (-1: none), or null
  const int32_t* tx_max_int; // [n_tx] depth to which each TX's tree is expanded, or null
  unsigned long long* stats;
  uint32_t* overflow;        // [0] largest node slot requested, [1] coarse slot requested
  uint32_t* err;             // [4] propagation: 1-4 a bounded wait gave up, >= 5 a self-check failed; details
  long long wait_limit;      // cycles after which a wait gives up; 0: each wait's default
  int rx_first;              // last level: test the reachable RXs' visibility before marching
};

// Self-checks of the propagation's indices (never expected to fail): the first failure
// writes its code and three details to err[0..3] (err[0] from zero by compare-and-swap)
// and the access it guards is skipped; the call then returns NIMBUS_ERR_STATE.
__device__ __forceinline__ void check_fail(const DTrace& tr, unsigned code, unsigned a, unsigned b, unsigned c) {
  if (tr.err && atomicCAS(tr.err, 0u, code) == 0u) {
    tr.err[1] = a;
    tr.err[2] = b;
    tr.err[3] = c;
  }
}

// The limit of a bounded wait: its default, or the context's test limit.
__device__ __forceinline__ long long wait_cap(const DTrace& tr, long long dflt) {
  return tr.wait_limit > 0 ? tr.wait_limit : dflt;
}

// Nodes of one level, structure of arrays (reflection and diffraction apart).
//   a: apex (reception point) xyz, IE index bits
//   b: incoming direction xyz, parent index bits
//   m: tx | nr << 16 | nd << 20 | depth << 24 | parent_is_diffraction << 28
struct NodeLevel {
  float4* ra;
  float4* rb;
  uint32_t* rm;
  float4* da;
  float4* db;
  uint32_t* dm;
  uint32_t* cnt;   // [0] reflection nodes, [1] diffraction nodes
  uint32_t cap_r, cap_d;
  // single-launch propagation only (null otherwise): per node slot, 1 once its record
  // is written; and the count of cone tasks created and not yet finished
  uint8_t* rdy_r;
  uint8_t* rdy_d;
  unsigned long long* outstanding;
};

struct CoarseBuf {
  uint4* rec;      // tx, rx, node ref (index | diffraction << 31), depth
  float* miss;
  uint32_t* cnt;
  uint32_t cap;
};

struct ConeD {
  float3 apex, axis;
  float sin_a, cos_a;
  int kind;
  float3 pn;               // reflection: oriented surface normal
  float3 tlo, thi, rmid;   // diffraction: separation planes and mid direction
  Endpoint origin;
};

// Separation planes (Section 2.2.4): reflections keep what lies more than sep_eps
// in front of the tangent plane at the apex; a diffracted ray keeps what lies
// between the planes half-way to its fan neighbours, on its own side of the edge.
__device__ __forceinline__ bool planes_ok(const ConeD& c, float3 q, float sep_eps) {
  float3 r = q - c.apex;
  if (c.kind == CONE_REFLECT) return dot(r, c.pn) > sep_eps;
  if (c.kind == CONE_DIFFRACT) return dot(r, c.tlo) >= 0.f && dot(r, c.thi) < 0.f && dot(r, c.rmid) > 0.f;
  return true;
}

__device__ __forceinline__ int rx_lower_bound(const DTrace& tr, uint64_t key) {
  int lo = 0, hi = tr.n_rx_sorted;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (tr.rx_sorted[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Voxel cone tracing of one cone (Section 2.2.4).  The axis is walked voxel by
// voxel; where the march distance is at most 1 the neighbouring voxels not yet
// evaluated for this cone are tested (voxel sphere, then each IE's subvoxel
// sphere, the separation planes, then acc's acceptance test).  A voxel whose march
// distance m >= 2 vouches for the (2(m-2)+1)^3 box around it, which the walk
// crosses without reading the field.  The cone stops after the first evaluation
// that accepted a point IE.
template <class Acc>
__device__ void march_cone(const DScene& s, const DTrace& tr, const ConeD& c, bool test_edges, bool want_all,
                           Acc& acc, unsigned long long& bytes, uint32_t& evals) {
  Walk w;
  walk_init(s, c.apex, c.axis, w);
  int last[3] = {0, 0, 0}, anchor[3] = {0, 0, 0};
  bool have_last = false;
  int rad = -1;
  const int max_steps = s.nx + s.ny + s.nz + 3;
  const float inf = __int_as_float(0x7f800000);
  for (int step = 0; step < max_steps; ++step) {
    bool in_box = rad >= 0 && abs(w.v[0] - anchor[0]) <= rad && abs(w.v[1] - anchor[1]) <= rad &&
                  abs(w.v[2] - anchor[2]) <= rad;
    if (!in_box) {
      long long ci = cell_index(s, w.v[0], w.v[1], w.v[2]);
      int m = tr.march[ci];
      bytes += 1;
      if (m > 1) {
        anchor[0] = w.v[0]; anchor[1] = w.v[1]; anchor[2] = w.v[2];
        rad = m - 2;
      } else {
        ++evals;
        bool stop = false;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int u0 = w.v[0] + dx, u1 = w.v[1] + dy, u2 = w.v[2] + dz;
              if (!in_grid(s, u0, u1, u2)) continue;
              if (have_last && abs(u0 - last[0]) <= 1 && abs(u1 - last[1]) <= 1 && abs(u2 - last[2]) <= 1) continue;
              long long cu = cell_index(s, u0, u1, u2);
              uint2 cell = __ldg(&s.cells[cu]);
              bool has_rx = (__ldg(&tr.rx_bits[cu >> 5]) >> (cu & 31)) & 1u;
              bytes += 12;
              if (cell.y == 0 && !has_rx) continue;
              if (!cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, voxel_center(s, u0, u1, u2), s.r_vox)) continue;
              for (uint32_t k = 0; k < cell.y; ++k) {
                uint32_t id = cell.x + k;
                const IERec* r = &s.ies[id];
                float4 nm = __ldg(&r->nrm_meta);
                float4 sc = __ldg(&r->sc_pc);
                bytes += 32;
                uint32_t kind = __float_as_uint(nm.w) & 1u;
                if (kind == IE_EDGE && !test_edges) continue;
                if (kind == IE_POINT && stop && !want_all) continue;
                if (!cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, xyz(sc), s.r_sub)) continue;
                float4 rp = __ldg(&r->rp_lab);
                bytes += 16;
                if (!planes_ok(c, xyz(rp), tr.sep_eps)) continue;
                if (acc.ie(id, xyz(rp), kind, __float_as_uint(rp.w), bytes) && kind == IE_POINT) stop = true;
              }
              if (has_rx) {
                for (int q = rx_lower_bound(tr, (uint64_t)cu << 32); q < tr.n_rx_sorted; ++q) {
                  uint64_t e = tr.rx_sorted[q];
                  bytes += 8;
                  if ((long long)(e >> 32) != cu) break;
                  int j = (int)(e & 0xffffffffu);
                  float3 pos = xyz(__ldg(&tr.rx[j]));
                  bytes += 16;
                  if (!cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, pos, s.r_sub)) continue;
                  if (!planes_ok(c, pos, tr.sep_eps)) continue;
                  float3 v = pos - c.apex;
                  float3 perp = v - dot(v, c.axis) * c.axis;
                  acc.rx(j, pos, len(perp), bytes);
                }
              }
            }
        have_last = true;
        last[0] = w.v[0]; last[1] = w.v[1]; last[2] = w.v[2];
        if (stop) break;
      }
    }
    if (!walk_next(s, w, inf)) break;
  }
}

// Transmission-phase acceptance: TX -> IE and TX -> RX visibility from the tables.
struct PrimaryAcc {
  const DTrace* tr;
  int t;
  uint32_t* first_bits;
  uint32_t* los;
  __device__ bool ie(uint32_t id, float3, uint32_t, uint32_t, unsigned long long& bytes) {
    size_t wi = (size_t)t * tr->ie_words + (id >> 5);
    uint32_t bit = 1u << (id & 31);
    bytes += 4;
    if (!(__ldg(&tr->vis_ie[wi]) & bit)) return false;
    if (!(first_bits[wi] & bit)) atomicOr(&first_bits[wi], bit);
    return true;
  }
  __device__ void rx(int j, float3, float miss, unsigned long long& bytes) {
    bytes += 4;
    if (tr->rx_owner && tr->rx_owner[j] >= 0 && tr->rx_owner[j] != t) return;
    if (__ldg(&tr->vis_rx[(size_t)t * tr->n_rx + j])) atomicMin(&los[(size_t)t * tr->n_rx + j], __float_as_uint(miss));
  }
};

__device__ __forceinline__ void add_stats(const DTrace& tr, uint32_t cones, uint32_t vis, unsigned long long bytes,
                                          uint32_t evals, uint32_t no_rx = 0) {
  // warp-aggregated counters
  unsigned long long c = cones, v = vis, b = bytes, e = evals, z = no_rx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&tr.stats[ST_CONES], c);
    atomicAdd(&tr.stats[ST_VIS], v);
    atomicAdd(&tr.stats[ST_BYTES], b);
    atomicAdd(&tr.stats[ST_EVALS], e);
    if (z) atomicAdd(&tr.stats[ST_NO_RX], z);
  }
}

// TX -> IE and TX -> RX visibility (the transmission phase's ray toward each IE).
__global__ void k_vis_tables(DScene s, DTrace tr) {
  const int64_t n_ie = s.n_ie;
  const int64_t per_tx = n_ie + tr.n_rx;
  const int64_t total = per_tx * tr.n_tx;
  unsigned long long bytes = 0;
  uint32_t vis = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(i / per_tx);
    int64_t k = i % per_tx;
    float3 T = xyz(tr.tx[t]);
    Endpoint none{IGN_NONE, NB_NONE_LABEL};
    ++vis;
    if (k < n_ie) {
      float4 rp = __ldg(&s.ies[k].rp_lab);
      uint32_t kind = __float_as_uint(__ldg(&s.ies[k].nrm_meta).w) & 1u;
      Endpoint eb{kind == IE_EDGE ? IGN_ANY : IGN_LABEL, __float_as_uint(rp.w)};
      if (visible(s, T, xyz(rp), none, eb, bytes))
        atomicOr(const_cast<uint32_t*>(&tr.vis_ie[(size_t)t * tr.ie_words + (k >> 5)]), 1u << (k & 31));
    } else {
      int j = (int)(k - n_ie);
      const_cast<uint32_t*>(tr.vis_rx)[(size_t)t * tr.n_rx + j] =
          visible(s, T, xyz(tr.rx[j]), none, none, bytes) ? 1u : 0u;
    }
  }
  add_stats(tr, 0, vis, bytes, 0);
}

// Uniform launch (transmission phase): Fibonacci-lattice cones from every TX.
__global__ void k_primary(DScene s, DTrace tr, uint32_t* first_bits, uint32_t* los) {
  const int64_t total = (int64_t)tr.n_tx * tr.n_launch;
  unsigned long long bytes = 0;
  uint32_t cones = 0, evals = 0;
  const bool test_edges = tr.max_int >= 1 && tr.max_diff >= 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(i / tr.n_launch);
    int64_t q = i % tr.n_launch;
    double z = 1.0 - (2.0 * (double)q + 1.0) / (double)tr.n_launch;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double phi = fmod((double)q * tr.golden, 2.0 * PI_D);
    double sp, cp;
    sincos(phi, &sp, &cp);
    ConeD c;
    c.apex = xyz(tr.tx[t]);
    c.axis = f3((float)(r * cp), (float)(r * sp), (float)z);
    c.sin_a = tr.sin_a0;
    c.cos_a = tr.cos_a0;
    c.kind = CONE_PRIMARY;
    c.origin = Endpoint{IGN_NONE, NB_NONE_LABEL};
    PrimaryAcc acc{&tr, t, first_bits, los};
    ++cones;
    march_cone(s, tr, c, test_edges, true, acc, bytes, evals);
  }
  add_stats(tr, cones, 0, bytes, evals);
}

// Depth-1 nodes: one per (TX, IE) accepted by any primary cone (a set), in IE order.
__global__ void k_first_flags(DScene s, DTrace tr, const uint32_t* first_bits, uint32_t* fr, uint32_t* fd) {
  const int64_t total = (int64_t)tr.n_tx * s.n_ie;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(i / s.n_ie);
    int64_t k = i % s.n_ie;
    bool hit = (first_bits[(size_t)t * tr.ie_words + (k >> 5)] >> (k & 31)) & 1u;
    uint32_t kind = __float_as_uint(s.ies[k].nrm_meta.w) & 1u;
    bool ok = hit && tr.max_int >= 1 && (!tr.tx_max_int || tr.tx_max_int[t] >= 1) &&
              (kind == IE_POINT ? tr.max_refl >= 1 : tr.max_diff >= 1);
    fr[i] = ok && kind == IE_POINT;
    fd[i] = ok && kind == IE_EDGE;
  }
}

__global__ void k_first_nodes(DScene s, DTrace tr, const uint32_t* fr, const uint32_t* pr, const uint32_t* fd,
                              const uint32_t* pd, NodeLevel L) {
  const int64_t total = (int64_t)tr.n_tx * s.n_ie;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (!fr[i] && !fd[i]) continue;
    int t = (int)(i / s.n_ie);
    uint32_t k = (uint32_t)(i % s.n_ie);
    float3 T = xyz(tr.tx[t]);
    float3 rp = xyz(s.ies[k].rp_lab);
    float3 e = normalize(rp - T);
    bool refl = fr[i] != 0;
    uint32_t slot = refl ? pr[i] : pd[i];
    uint32_t cap = refl ? L.cap_r : L.cap_d;
    if (slot >= cap) {
      atomicMax(&tr.overflow[0], slot + 1);
      continue;
    }
    uint32_t meta = (uint32_t)t | ((refl ? 1u : 0u) << 16) | ((refl ? 0u : 1u) << 20) | (1u << 24);
    float4 a = make_float4(rp.x, rp.y, rp.z, __uint_as_float(k));
    float4 b = make_float4(e.x, e.y, e.z, __uint_as_float(NO_NODE));
    if (refl) {
      L.ra[slot] = a; L.rb[slot] = b; L.rm[slot] = meta;
    } else {
      L.da[slot] = a; L.db[slot] = b; L.dm[slot] = meta;
    }
  }
}

__global__ void k_first_counts(const uint32_t* tot_r, const uint32_t* tot_d, NodeLevel L) {
  L.cnt[0] = min(*tot_r, L.cap_r);
  L.cnt[1] = min(*tot_d, L.cap_d);
}

__device__ __forceinline__ void emit_coarse(const DTrace& tr, CoarseBuf& cb, uint32_t t, uint32_t j, uint32_t node,
                                            uint32_t depth, float miss) {
  if (t >= (uint32_t)tr.n_tx || j >= (uint32_t)tr.n_rx) {
    check_fail(tr, 11u, t, j, node);
    return;
  }
  uint32_t slot = atomicAdd(cb.cnt, 1u);
  if (slot >= cb.cap) {
    atomicMax(&tr.overflow[1], slot + 1);
    return;
  }
  cb.rec[slot] = make_uint4(t, j, node, depth);
  cb.miss[slot] = miss;
}

// LOS of the paper's launch (a ray toward each RX): every RX visible from the TX,
// at miss distance 0 (the ray points at the RX).
__global__ void k_los_from_vis(DTrace tr, uint32_t* los) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)tr.n_tx * tr.n_rx) return;
  const int t = (int)(i / tr.n_rx), j = (int)(i % tr.n_rx);
  if (tr.rx_owner && tr.rx_owner[j] >= 0 && tr.rx_owner[j] != t) return;
  if (tr.vis_rx[i]) los[i] = __float_as_uint(0.f);
}

// LOS coarse paths: RXs reached by a primary cone.
__global__ void k_los(DTrace tr, const uint32_t* los, CoarseBuf cb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tr.n_tx * tr.n_rx) return;
  uint32_t m = los[i];
  if (m != 0xFFFFFFFFu) emit_coarse(tr, cb, i / tr.n_rx, i % tr.n_rx, NO_NODE, 0, __uint_as_float(m));
}

// A child node of the next level (Section 2.2.3): the accepted IE becomes the apex
// of a reflected cone (point IE) or of a Keller fan (edge IE).
__device__ void emit_child(const DTrace& tr, NodeLevel& next, uint32_t id, float3 rp, float3 apex, uint32_t kind,
                           uint32_t tx, uint32_t nr, uint32_t nd, uint32_t depth, uint32_t self_ref) {
  if (id >= tr.n_ie || kind > IE_EDGE || tx >= (uint32_t)tr.n_tx) {
    check_fail(tr, 10u, id, kind, tx);
    return;
  }
  const uint32_t cnr = nr + (kind == IE_POINT), cnd = nd + (kind == IE_EDGE);
  if ((int)cnr > tr.max_refl || (int)cnd > tr.max_diff) return;
  const bool refl = kind == IE_POINT;
  const uint32_t slot = atomicAdd(&next.cnt[refl ? 0 : 1], 1u);
  const uint32_t cap = refl ? next.cap_r : next.cap_d;
  if (slot >= cap) {
    atomicMax(&tr.overflow[0], slot + 1);
    return;
  }
  const float3 e = normalize(rp - apex);
  const uint32_t meta = tx | (cnr << 16) | (cnd << 20) | ((depth + 1) << 24) | ((self_ref >> 31) << 28);
  const float4 a = make_float4(rp.x, rp.y, rp.z, __uint_as_float(id));
  const float4 b = make_float4(e.x, e.y, e.z, __uint_as_float(self_ref & 0x7fffffffu));
  if (refl) {
    next.ra[slot] = a; next.rb[slot] = b; next.rm[slot] = meta;
  } else {
    next.da[slot] = a; next.db[slot] = b; next.dm[slot] = meta;
  }
  if (next.outstanding) {
    // single launch: count the child's cone tasks before publishing the record, so
    // that the count cannot reach zero while this warp may still create work
    atomicAdd(next.outstanding, refl ? 1ull : (unsigned long long)tr.M);
    __threadfence();
    *(volatile uint8_t*)(refl ? next.rdy_r + slot : next.rdy_d + slot) = 1;
  }
}

// What one propagation cone needs besides its geometry.
struct LevelCone {
  uint32_t tx, nr, nd, depth, self_ref;
  bool can_child, test_edges;
};

// The candidates of one evaluation of a cone (IEs and RXs in its accepted voxels)
// wait in the warp's slot of its block's board, in the order the cone met them, so
// that the warps of the block that have no cone left can walk some of their
// visibility rays: the rays of one evaluation are independent, and a cone that meets
// hundreds of occluded candidates otherwise keeps one warp busy for tens of
// milliseconds after the rest of its launch has finished.  A ray is walked by one
// whole warp whichever warp takes it, so every decision is the same.
//   word: generation << 24 | entries << 12 | entries taken; a warp takes entry k
//   with a compare-and-swap of the word (a stale generation fails).
// Ordering: the owner's lanes store the entries, a __syncwarp orders them before
// lane 0's fence and the exchange that publishes the word, and a taker fences after
// its compare-and-swap before reading an entry.  Every board word that steers a warp
// (the word, first_vis, done) is read by lane 0 and broadcast, so that no warp splits
// around the whole-warp walk.
// At the last level a point IE only decides whether the cone stops, and the walk in
// order skips the point IEs after the first visible one.  Here an entry is skipped
// once a visible point IE with a smaller index is known (first_vis); the owner then
// counts the rays and bytes of exactly the entries the walk in order tests, and no
// entry before the first visible one can have been skipped.
#ifndef HELP_CAP
#define HELP_CAP 64
#endif
constexpr uint32_t CAND_RX = 2;
struct HelpSlot {
  unsigned word;
  unsigned done;        // entries walked or skipped
  unsigned first_vis;   // smallest index (within the evaluation) of a visible point IE
  unsigned qbase;       // index of entry 0 within the evaluation
  float4 h0;            // cone apex, origin label bits
  uint4 h1;             // origin mode, tx | nr << 16 | nd << 20 | depth << 24, self_ref, can_child
  float4 a[HELP_CAP];   // target, IE or RX index bits
  uint2 b[HELP_CAP];    // kind (IE_POINT, IE_EDGE, CAND_RX), label or miss bits
  unsigned r[HELP_CAP]; // bit 31: walked; the walk's bytes
};

// Walk entry t of slot H (any warp of the block, all lanes).
__device__ __forceinline__ void help_walk(const DScene& s, const DTrace& tr, NodeLevel& next, CoarseBuf& cb,
                                          HelpSlot& H, unsigned t, int lane) {
  const float4 a = H.a[t];
  const uint2 b = H.b[t];
  const float4 h0 = H.h0;
  const uint4 h1 = H.h1;
  const unsigned q = H.qbase + t;
  const bool can_child = h1.w != 0;
  unsigned r = 0;
  const uint32_t id = __float_as_uint(a.w);
  bool bad = b.x > CAND_RX || (b.x == CAND_RX ? id >= (uint32_t)tr.n_rx : id >= tr.n_ie);
  if (!bad && b.x != CAND_RX) bad = (__float_as_uint(__ldg(&s.ies[id].nrm_meta).w) & 1u) != b.x;
  // the skip must be the same on every lane (the walk below is a whole-warp walk), but
  // other warps lower first_vis concurrently: lane 0 reads it once for the warp
  unsigned fv = 0xffffffffu;
  if (lane == 0) fv = *(volatile unsigned*)&H.first_vis;
  fv = __shfl_sync(FULL, fv, 0);
  if (bad) {   // an entry that was not what its owner stored (never expected)
    if (lane == 0) check_fail(tr, 8u, id, b.x, t);
  } else if (!(b.x == IE_POINT && !can_child && fv < q)) {
    unsigned long long by = 0;
    const float3 apex = xyz(h0), tgt = xyz(a);
    const Endpoint origin{(int)h1.x, __float_as_uint(h0.w)};
    const Endpoint eb = b.x == CAND_RX ? Endpoint{IGN_NONE, NB_NONE_LABEL}
                                       : Endpoint{b.x == IE_EDGE ? IGN_ANY : IGN_LABEL, b.y};
    const bool v = visible_warp(s, apex, tgt, origin, eb, lane, by);
    r = (1u << 31) | min(__reduce_add_sync(FULL, (unsigned)by), 0x7fffffffu);
    if (v && lane == 0) {
      const uint32_t m = h1.y, tx = m & 0xffffu, nr = (m >> 16) & 0xfu, nd = (m >> 20) & 0xfu, dep = (m >> 24) & 0xfu;
      if (b.x == CAND_RX) {
        emit_coarse(tr, cb, tx, __float_as_uint(a.w), h1.z, dep, __uint_as_float(b.y));
      } else {
        if (can_child) emit_child(tr, next, __float_as_uint(a.w), tgt, apex, b.x, tx, nr, nd, dep, h1.z);
        if (b.x == IE_POINT) atomicMin(&H.first_vis, q);
      }
    }
  }
  if (lane == 0) {
    H.r[t] = r;
    __threadfence_block();
    atomicAdd(&H.done, 1u);
  }
  __syncwarp();
}

// Take the next entry of slot H: lane 0 claims it, every lane gets its index, or
// 0xffffffff when every entry is taken.
__device__ __forceinline__ unsigned help_take(HelpSlot& H, int lane) {
  unsigned tk = 0xffffffffu;
  if (lane == 0) {
    unsigned w = *(volatile unsigned*)&H.word;
    while (((w >> 12) & 0xfffu) > (w & 0xfffu)) {
      const unsigned o = atomicCAS(&H.word, w, w + 1);
      if (o == w) {
        tk = w & 0xfffu;
        __threadfence_block();   // acquire: the entries were published before the word
        break;
      }
      w = o;
    }
  }
  tk = __shfl_sync(FULL, tk, 0);
  __syncwarp();
  return tk;
}

// The owner's side: publish the hn entries collected, walk them together with any
// idle warps of the block, wait until all are done, close the slot, and count the
// rays and bytes the walk in order would have.  The slot keeps, across the batches
// of one evaluation, the first visible point IE so far (first_vis) and the entries
// already walked (qbase); the owner resets both when an evaluation starts.
__device__ __forceinline__ void help_flush(const DScene& s, const DTrace& tr, NodeLevel& next, CoarseBuf& cb,
                                           HelpSlot& H, int& hn, int lane, unsigned long long& bytes, uint32_t& vis) {
  if (hn == 0) return;
  // the entries were stored by the lanes that found them: order every lane's stores
  // before lane 0's fence and the publishing exchange, so that a warp that takes an
  // entry reads what was stored, not what the slot held before
  __syncwarp();
  // the generation lives in the slot's word; only its owner changes it (lane 0 uses it)
  const unsigned gen = lane == 0 ? *(volatile unsigned*)&H.word >> 24 : 0u;
  if (lane == 0) {
    H.done = 0;
    __threadfence_block();
    atomicExch(&H.word, (gen << 24) | ((unsigned)hn << 12));
  }
  __syncwarp();
  for (;;) {
    const unsigned tk = help_take(H, lane);
    if (tk == 0xffffffffu) break;
    help_walk(s, tr, next, cb, H, tk, lane);
  }
  if (lane == 0) {
    // entries taken by other warps: each is one visibility ray, at most milliseconds
    const long long t0 = clock64();
    while (*(volatile unsigned*)&H.done < (unsigned)hn) {
      if (clock64() - t0 > wait_cap(tr, 4000000000ll)) {
        atomicExch(tr.err, 3u);
        break;
      }
      __nanosleep(32);
    }
    __threadfence_block();
    atomicExch(&H.word, ((gen + 1) & 0xffu) << 24);
  }
  __syncwarp();
  const unsigned Fn = __shfl_sync(FULL, lane == 0 ? *(volatile unsigned*)&H.first_vis : 0u, 0), qn = H.qbase;
  const bool can_child = H.h1.w != 0;
  for (int t0 = 0; t0 < hn; t0 += 32) {
    const int t = t0 + lane;
    bool counted = false;
    if (t < hn) {
      const unsigned r = H.r[t];
      counted = (r >> 31) && (can_child || H.b[t].x != IE_POINT || qn + (unsigned)t <= Fn);
      if (counted) bytes += r & 0x7fffffffu;
    }
    const unsigned cm = __ballot_sync(FULL, counted);
    if (lane == 0) vis += __popc(cm);
  }
  __syncwarp();
  if (lane == 0) H.qbase = qn + (unsigned)hn;
  hn = 0;
  __syncwarp();
}

// Voxel cone tracing of one propagation cone by a whole warp (Section 2.2.4).  The
// walk along the axis is the same on every lane.  At an evaluation lane l < 27
// tests neighbour voxel l (already-evaluated voxels skipped, voxel sphere vs cone);
// the IEs of each accepted voxel are screened one per lane (subvoxel sphere, kind,
// separation planes), and each candidate's visibility ray (Section 2.2.1) is then
// walked by the whole warp with the Eq. 1 sums split across lanes.  Visible IEs
// become children; RXs reached become coarse paths; the cone stops after the
// evaluation in which a point IE was visible.  Without children to emit (last
// level) the remaining point IEs of that evaluation are not tested: they can only
// confirm the stop.
template <bool HELP>
__device__ void march_cone_warp(const DScene& s, const DTrace& tr, const ConeD& c, const LevelCone& lc,
                                NodeLevel& next, CoarseBuf& cb, HelpSlot* Hp, float t_end, int lane,
                                unsigned long long& bytes, uint32_t& evals, uint32_t& vis) {
  if constexpr (HELP) {
    HelpSlot& H = *Hp;
    if (lane == 0) {
      // no entry of this slot is out (the last batch was waited for): the header is free
      H.h0 = make_float4(c.apex.x, c.apex.y, c.apex.z, __uint_as_float(c.origin.label));
      H.h1 = make_uint4((unsigned)c.origin.mode, lc.tx | (lc.nr << 16) | (lc.nd << 20) | (lc.depth << 24),
                        lc.self_ref, lc.can_child ? 1u : 0u);
    }
    __syncwarp();
  }
  const unsigned lt = (1u << lane) - 1u;
  Walk w;
  walk_init(s, c.apex, c.axis, w);
  int last[3] = {0, 0, 0}, anchor[3] = {0, 0, 0};
  bool have_last = false;
  int rad = -1;
  const int max_steps = s.nx + s.ny + s.nz + 3;
  const int ldx = lane % 3 - 1, ldy = (lane / 3) % 3 - 1, ldz = lane / 9 - 1;   // lanes 0..26
  for (int step = 0; step < max_steps; ++step) {
    const bool in_box = rad >= 0 && abs(w.v[0] - anchor[0]) <= rad && abs(w.v[1] - anchor[1]) <= rad &&
                        abs(w.v[2] - anchor[2]) <= rad;
    if (!in_box) {
      const int m = tr.march[cell_index(s, w.v[0], w.v[1], w.v[2])];
      if (lane == 0) bytes += 1;
      if (m > 1) {
        anchor[0] = w.v[0]; anchor[1] = w.v[1]; anchor[2] = w.v[2];
        rad = m - 2;
      } else {
        if (lane == 0) ++evals;
        bool ok = false, has_rx = false;
        uint2 cell = make_uint2(0u, 0u);
        long long cu = 0;
        if (lane < 27) {
          const int u0 = w.v[0] + ldx, u1 = w.v[1] + ldy, u2 = w.v[2] + ldz;
          const bool seen = have_last && abs(u0 - last[0]) <= 1 && abs(u1 - last[1]) <= 1 && abs(u2 - last[2]) <= 1;
          if (in_grid(s, u0, u1, u2) && !seen) {
            cu = cell_index(s, u0, u1, u2);
            cell = __ldg(&s.cells[cu]);
            has_rx = (__ldg(&tr.rx_bits[cu >> 5]) >> (cu & 31)) & 1u;
            bytes += 12;
            ok = (cell.y > 0 || has_rx) &&
                 cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, voxel_center(s, u0, u1, u2), s.r_vox);
          }
        }
        bool stop;
        if constexpr (HELP) {
          HelpSlot& H = *Hp;
          // Collect the evaluation's candidates in the order the walk in order meets them
          // (IE voxels by lane, their IEs in chunks of 32, then the RX voxels' runs)
          // until the slot is full, walk that batch, and go on from where collecting
          // stopped (the chunk that did not fit is screened again; its bytes count once).
          int hn = 0;                  // entries collected and not yet walked
          if (lane == 0) {
            H.first_vis = 0xffffffffu;
            H.qbase = 0;
          }
          unsigned vm = __ballot_sync(FULL, ok && cell.y > 0);   // IE voxels left
          unsigned rm = __ballot_sync(FULL, ok && has_rx);       // RX voxels left (never stop the cone)
          uint32_t k0 = 0;             // next IE chunk of voxel ffs(vm)
          int qb = -1;                 // next RX chunk of voxel ffs(rm); -1 before its first
          for (;;) {
            bool full = false;
            while (vm) {
              const int src = __ffs(vm) - 1;
              const uint32_t base = __shfl_sync(FULL, cell.x, src), cnt = __shfl_sync(FULL, cell.y, src);
              if (k0 >= cnt) {
                vm &= vm - 1;
                k0 = 0;
                continue;
              }
              const uint32_t k = k0 + lane, id = base + k;
              bool cand = false;
              uint32_t kind = IE_POINT, lbl = 0;
              float3 rp = f3(0.f, 0.f, 0.f);
              unsigned by = 0;
              if (k < cnt) {
                const IERec* r = &s.ies[id];
                const float4 nm = __ldg(&r->nrm_meta), sc = __ldg(&r->sc_pc);
                by += 32;
                kind = __float_as_uint(nm.w) & 1u;
                if ((kind == IE_POINT || lc.test_edges) && cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, xyz(sc), s.r_sub)) {
                  const float4 q = __ldg(&r->rp_lab);
                  by += 16;
                  rp = xyz(q);
                  lbl = __float_as_uint(q.w);
                  cand = planes_ok(c, rp, tr.sep_eps);
                }
              }
              const unsigned cm = __ballot_sync(FULL, cand);
              if (hn + __popc(cm) > HELP_CAP) {
                full = true;
                break;
              }
              if (cand) {
                const int k2 = hn + __popc(cm & lt);
                H.a[k2] = make_float4(rp.x, rp.y, rp.z, __uint_as_float(id));
                H.b[k2] = make_uint2(kind, lbl);
              }
              hn += __popc(cm);
              bytes += by;
              k0 += 32;
            }
            while (!full && !vm && rm) {
              const int src = __ffs(rm) - 1;
              const long long cus = __shfl_sync(FULL, cu, src);
              if (qb < 0) qb = rx_lower_bound(tr, (uint64_t)cus << 32);
              const int q = qb + lane;
              bool in = false, cand = false;
              int rj = 0;
              float3 pos = f3(0.f, 0.f, 0.f);
              float miss = 0.f;
              unsigned by = 0;
              if (q < tr.n_rx_sorted) {
                const uint64_t e = tr.rx_sorted[q];
                by += 8;
                in = (long long)(e >> 32) == cus;
                if (in) {
                  rj = (int)(e & 0xffffffffu);
                  pos = xyz(__ldg(&tr.rx[rj]));
                  by += 16;
                  cand = cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, pos, s.r_sub) && planes_ok(c, pos, tr.sep_eps) &&
                         !(tr.rx_owner && tr.rx_owner[rj] >= 0 && (uint32_t)tr.rx_owner[rj] != lc.tx) &&
                         !(tr.rx_max_int && tr.rx_max_int[rj] >= 0 && (int)lc.depth > tr.rx_max_int[rj]);
                  if (cand) {
                    const float3 v = pos - c.apex;
                    miss = len(v - dot(v, c.axis) * c.axis);
                  }
                }
              }
              const unsigned inm = __ballot_sync(FULL, in);
              const unsigned cm = __ballot_sync(FULL, cand);
              if (hn + __popc(cm) > HELP_CAP) {
                full = true;
                break;
              }
              if (cand) {
                const int k2 = hn + __popc(cm & lt);
                H.a[k2] = make_float4(pos.x, pos.y, pos.z, __uint_as_float((uint32_t)rj));
                H.b[k2] = make_uint2(CAND_RX, __float_as_uint(miss));
              }
              hn += __popc(cm);
              bytes += by;
              if (inm != FULL) {   // the voxel's RX run ended in this chunk
                rm &= rm - 1;
                qb = -1;
              } else {
                qb += 32;
              }
            }
            help_flush(s, tr, next, cb, H, hn, lane, bytes, vis);
            if (!full) break;
          }
          // a point IE of this evaluation was visible
          stop = __shfl_sync(FULL, lane == 0 ? *(volatile unsigned*)&H.first_vis : 0u, 0) != 0xffffffffu;
        } else {
          // each candidate walked at once by this warp
          stop = false;
          unsigned vm = __ballot_sync(FULL, ok && cell.y > 0);
          while (vm) {
            const int src = __ffs(vm) - 1;
            vm &= vm - 1;
            const uint32_t base = __shfl_sync(FULL, cell.x, src), cnt = __shfl_sync(FULL, cell.y, src);
            for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
              const uint32_t k = k0 + lane, id = base + k;
              bool cand = false;
              uint32_t kind = IE_POINT, lbl = 0;
              float3 rp = f3(0.f, 0.f, 0.f);
              if (k < cnt) {
                const IERec* r = &s.ies[id];
                const float4 nm = __ldg(&r->nrm_meta), sc = __ldg(&r->sc_pc);
                bytes += 32;
                kind = __float_as_uint(nm.w) & 1u;
                if ((kind == IE_POINT || lc.test_edges) && cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, xyz(sc), s.r_sub)) {
                  const float4 q = __ldg(&r->rp_lab);
                  bytes += 16;
                  rp = xyz(q);
                  lbl = __float_as_uint(q.w);
                  cand = planes_ok(c, rp, tr.sep_eps);
                }
              }
              unsigned cm = __ballot_sync(FULL, cand);
              while (cm) {
                const int j = __ffs(cm) - 1;
                cm &= cm - 1;
                const uint32_t cid = __shfl_sync(FULL, id, j), ckind = __shfl_sync(FULL, kind, j);
                const uint32_t clab = __shfl_sync(FULL, lbl, j);
                const float3 crp = f3(__shfl_sync(FULL, rp.x, j), __shfl_sync(FULL, rp.y, j), __shfl_sync(FULL, rp.z, j));
                if (ckind == IE_POINT && stop && !lc.can_child) continue;
                if (lane == 0) ++vis;
                const Endpoint eb{ckind == IE_EDGE ? IGN_ANY : IGN_LABEL, clab};
                if (!visible_warp(s, c.apex, crp, c.origin, eb, lane, bytes)) continue;
                if (lc.can_child && lane == 0)
                  emit_child(tr, next, cid, crp, c.apex, ckind, lc.tx, lc.nr, lc.nd, lc.depth, lc.self_ref);
                if (ckind == IE_POINT) stop = true;
              }
            }
          }
          // RXs in the accepted voxels (never stop the cone)
          unsigned rm = __ballot_sync(FULL, ok && has_rx);
          while (rm) {
            const int src = __ffs(rm) - 1;
            rm &= rm - 1;
            const long long cus = __shfl_sync(FULL, cu, src);
            const int q0 = rx_lower_bound(tr, (uint64_t)cus << 32);
            for (int qb = q0;; qb += 32) {
              const int q = qb + lane;
              bool in = false, cand = false;
              int rj = 0;
              float3 pos = f3(0.f, 0.f, 0.f);
              float miss = 0.f;
              if (q < tr.n_rx_sorted) {
                const uint64_t e = tr.rx_sorted[q];
                bytes += 8;
                in = (long long)(e >> 32) == cus;
                if (in) {
                  rj = (int)(e & 0xffffffffu);
                  pos = xyz(__ldg(&tr.rx[rj]));
                  bytes += 16;
                  cand = cone_sphere(c.apex, c.axis, c.sin_a, c.cos_a, pos, s.r_sub) && planes_ok(c, pos, tr.sep_eps) &&
                         !(tr.rx_owner && tr.rx_owner[rj] >= 0 && (uint32_t)tr.rx_owner[rj] != lc.tx) &&
                         !(tr.rx_max_int && tr.rx_max_int[rj] >= 0 && (int)lc.depth > tr.rx_max_int[rj]);
                  if (cand) {
                    const float3 v = pos - c.apex;
                    miss = len(v - dot(v, c.axis) * c.axis);
                  }
                }
              }
              const unsigned inm = __ballot_sync(FULL, in);
              unsigned cm = __ballot_sync(FULL, cand);
              while (cm) {
                const int j = __ffs(cm) - 1;
                cm &= cm - 1;
                const int crj = __shfl_sync(FULL, rj, j);
                const float cmiss = __shfl_sync(FULL, miss, j);
                const float3 cpos = f3(__shfl_sync(FULL, pos.x, j), __shfl_sync(FULL, pos.y, j), __shfl_sync(FULL, pos.z, j));
                if (lane == 0) ++vis;
                if (visible_warp(s, c.apex, cpos, c.origin, Endpoint{IGN_NONE, NB_NONE_LABEL}, lane, bytes) && lane == 0)
                  emit_coarse(tr, cb, lc.tx, (uint32_t)crj, lc.self_ref, lc.depth, cmiss);
              }
              if (inm != FULL) break;   // the voxel's RX run ended in this chunk
            }
          }
        }
        have_last = true;
        last[0] = w.v[0]; last[1] = w.v[1]; last[2] = w.v[2];
        if (stop) break;
      }
    }
    if (!walk_next(s, w, t_end)) break;
  }
}

// The RXs that could pass the RX screening of this cone's march (march_cone_warp):
// the same cone-sphere, separation-plane, owner and depth tests, each loosened by
// 1e-5 (|v| + 1) m (|v|: the RX's distance from the apex), ten times the FP32 error of
// the screening's dot products at these distances, so that no RX the screening could
// accept is rejected here.  Returns the largest axial distance dot(v, axis) among
// them, or -1 when there is none (every lane gets the same value).  A cone that can
// emit no child (the last level) produces nothing but coarse paths to such RXs: with
// none its march is skipped, else the march stops once its walk is past the farthest
// (an RX is screened from walk voxels within one voxel of its own, whose axis points
// lie at most 2 sqrt(3) voxel edges further along the axis).
#ifndef NO_RX_MAX
#define NO_RX_MAX 4096
#endif
__device__ __forceinline__ bool rx_could_pass(const DScene& s, const DTrace& tr, const ConeD& c, const LevelCone& lc,
                                              int j, float* axial = nullptr) {
  if (tr.rx_owner && tr.rx_owner[j] >= 0 && (uint32_t)tr.rx_owner[j] != lc.tx) return false;
  if (tr.rx_max_int && tr.rx_max_int[j] >= 0 && (int)lc.depth > tr.rx_max_int[j]) return false;
  const float r = s.r_sub, r2 = r * r;
  const float3 v = xyz(__ldg(&tr.rx[j])) - c.apex;
  const float d2 = dot(v, v), tol = 1e-5f * (sqrtf(d2) + 1.f);
  bool in = d2 <= r2 * 1.001f + 1e-6f ||
            dot(v, c.axis) + r * c.sin_a + tol >= c.cos_a * sqrtf(fmaxf(d2 - r2, 0.f));
  if (in) {
    if (c.kind == CONE_REFLECT) in = dot(v, c.pn) > tr.sep_eps - tol;
    else if (c.kind == CONE_DIFFRACT)
      in = dot(v, c.tlo) >= -tol && dot(v, c.thi) < tol && dot(v, c.rmid) > -tol;
  }
  if (in && axial) *axial = fmaxf(dot(v, c.axis) + tol, 0.f);
  return in;
}

__device__ __forceinline__ float rx_reach(const DScene& s, const DTrace& tr, const ConeD& c, const LevelCone& lc,
                                          int lane) {
  float far = -1.f;
  for (int j = lane; j < tr.n_rx; j += 32) {
    float t;
    if (rx_could_pass(s, tr, c, lc, j, &t)) far = fmaxf(far, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) far = fmaxf(far, __shfl_xor_sync(FULL, far, o));
  return far;
}

// One propagation cone of level `cur`: the reflected cone of node idx (refl) or cone
// j of the Keller fan of diffraction node idx.
template <bool HELP>
__device__ __forceinline__ void level_cone(const DScene& s, const DTrace& tr, const NodeLevel& cur, NodeLevel& next,
                                           CoarseBuf& cb, HelpSlot* H, bool refl, uint32_t idx, int j, int lane,
                                           unsigned long long& bytes, uint32_t& cones, uint32_t& evals,
                                           uint32_t& vis, uint32_t& no_rx) {
  const float4 a = refl ? cur.ra[idx] : cur.da[idx];
  const float4 b = refl ? cur.rb[idx] : cur.db[idx];
  const uint32_t meta = refl ? cur.rm[idx] : cur.dm[idx];
  const uint32_t ie = __float_as_uint(a.w);
  if (ie >= (uint32_t)s.n_ie) {   // a node record the level did not write (never expected)
    if (lane == 0) check_fail(tr, 5u, ie, idx, refl ? 0u : 1u);
    return;
  }
  const IERec* r = &s.ies[ie];
  const float4 nm = __ldg(&r->nrm_meta);
  if ((__float_as_uint(nm.w) & 1u) != (refl ? (uint32_t)IE_POINT : (uint32_t)IE_EDGE) ||
      (!refl && __float_as_uint(__ldg(&r->bbc_pb).w) >= tr.n_edges)) {   // node kind and IE kind disagree
    if (lane == 0) check_fail(tr, 6u, ie, idx, (refl ? 0u : 1u) | ((__float_as_uint(nm.w) & 1u) << 1));
    return;
  }
  const uint32_t label = __float_as_uint(__ldg(&r->rp_lab).w);
  if (lane == 0) bytes += 32 + 36;
  const float3 e = xyz(b);
  ConeD c;
  c.apex = xyz(a);
  c.sin_a = tr.sin_a;
  c.cos_a = tr.cos_a;
  if (refl) {
    float3 n = xyz(nm);
    if (dot(n, e) > 0.f) n = -1.f * n;
    c.kind = CONE_REFLECT;
    c.axis = normalize(e - (2.f * dot(e, n)) * n);
    c.pn = n;
    c.origin = Endpoint{IGN_LABEL, label};
  } else {
    const double* E = s.edges + 12 * __float_as_uint(__ldg(&r->bbc_pb).w);
    if (lane == 0) bytes += 96;
    const float3 w = normalize(f3((float)(E[3] - E[0]), (float)(E[4] - E[1]), (float)(E[5] - E[2])));
    const float cb_ = dot(e, w);
    const float sb2 = 1.f - cb_ * cb_;
    if (sb2 < 1e-12f) return;
    const float sb = sqrtf(sb2);
    float3 ua, va;
    onb(w, &ua, &va);
    const float phi = (float)j * tr.dphi;
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float3 rr = cp * ua + sp * va;
    const float3 d = cb_ * w + sb * rr;
    const float3 n0 = f3((float)E[6], (float)E[7], (float)E[8]), n1 = f3((float)E[9], (float)E[10], (float)E[11]);
    if (!(dot(d, n0) > 0.f || dot(d, n1) > 0.f)) return;
    float slo, clo, shi, chi;
    sincosf(phi - 0.5f * tr.dphi, &slo, &clo);
    sincosf(phi + 0.5f * tr.dphi, &shi, &chi);
    c.kind = CONE_DIFFRACT;
    c.axis = normalize(d);
    c.tlo = (-slo) * ua + clo * va;
    c.thi = (-shi) * ua + chi * va;
    c.rmid = rr;
    c.origin = Endpoint{IGN_ANY, label};
  }
  LevelCone lc;
  lc.depth = (meta >> 24) & 0xfu;
  lc.nr = (meta >> 16) & 0xfu;
  lc.nd = (meta >> 20) & 0xfu;
  lc.tx = meta & 0xffffu;
  lc.self_ref = idx | (refl ? 0u : 0x80000000u);
  lc.can_child = (int)lc.depth < tr.max_int && (!tr.tx_max_int || (int)lc.depth < tr.tx_max_int[lc.tx]);
  lc.test_edges = lc.can_child && (int)lc.nd < tr.max_diff;
  if (lane == 0) ++cones;
  float t_end = __int_as_float(0x7f800000);
  if (!lc.can_child && tr.n_rx <= NO_RX_MAX) {
    const float far = rx_reach(s, tr, c, lc, lane);
    if (far < 0.f) {
      if (lane == 0) ++no_rx;
      return;
    }
    t_end = far + 4.f * s.h + 0.01f;
    // With rx_first: an RX is emitted only if it also sees the apex (the screening's
    // visibility ray: apex to RX, the cone's origin ignored, nothing at the RX).  When
    // none of the RXs that could pass the screening does, the cone emits nothing
    // whatever its march finds, so the march (and its point IEs' rays, which only
    // decide where it stops) is skipped.  The rays are the screening's own call with
    // the same arguments.  It pays where few reachable RXs are visible (an indoor
    // scan), not where many are (a street of a thousand RXs): a layout choice.
    bool seen = !tr.rx_first;
    for (int j0 = 0; j0 < tr.n_rx && !seen; j0 += 32) {
      const int j = j0 + lane;
      unsigned m = __ballot_sync(FULL, j < tr.n_rx && rx_could_pass(s, tr, c, lc, j));
      while (m && !seen) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        if (lane == 0) ++vis;
        seen = visible_warp(s, c.apex, xyz(__ldg(&tr.rx[j0 + src])), c.origin, Endpoint{IGN_NONE, NB_NONE_LABEL},
                            lane, bytes);
      }
    }
    if (!seen) {
      if (lane == 0) ++no_rx;
      return;
    }
  }
  march_cone_warp<HELP>(s, tr, c, lc, next, cb, H, t_end, lane, bytes, evals, vis);
}

// One propagation level: the reflected cones and Keller-fan cones of every node,
// one warp per cone, cones handed out by a counter (their costs differ widely).
// With HELP, a warp with no cone left walks visibility rays of its block's running
// cones (the board above) until every warp of the block has finished; the board (one
// slot per warp) is the launch's dynamic shared memory.  Without it each warp walks
// its own cones' rays as it meets them (the board's lists cost a little register
// room and time where no cone runs long).  Blocks of 128, 256 or 512 threads, all at
// 128 registers a thread (16 warps per SM).
#ifndef LEVEL_MAX_THREADS
#define LEVEL_MAX_THREADS 512
#endif
#ifndef LEVEL_MIN_BLOCKS
#define LEVEL_MIN_BLOCKS 1
#endif
template <bool HELP>
__global__ void __launch_bounds__(LEVEL_MAX_THREADS, LEVEL_MIN_BLOCKS) k_level(DScene s, DTrace tr, NodeLevel cur, NodeLevel next, CoarseBuf cb,
                                               unsigned long long* next_task) {
  extern __shared__ HelpSlot board[];
  __shared__ unsigned s_active;   // warps of the block still taking cones
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (HELP) {
    if (lane == 0) {
      board[wib].word = 0;
      board[wib].done = 0;
    }
    if (threadIdx.x == 0) s_active = (unsigned)nw;
    __syncthreads();
  }
  const uint32_t n_r = min(cur.cnt[0], cur.cap_r), n_d = min(cur.cnt[1], cur.cap_d);
  const int64_t total = (int64_t)n_r + (int64_t)n_d * tr.M;
  unsigned long long bytes = 0;
  uint32_t cones = 0, vis = 0, evals = 0, no_rx = 0;
  for (;;) {
    unsigned long long grab = 0;
    if (lane == 0) grab = atomicAdd(next_task, 1ull);
    const int64_t task = (int64_t)__shfl_sync(FULL, grab, 0);
    if (task >= total) break;
    const bool refl = task < n_r;
    const uint32_t idx = refl ? (uint32_t)task : (uint32_t)((task - n_r) / tr.M);
    const int j = refl ? 0 : (int)((task - n_r) % tr.M);
    level_cone<HELP>(s, tr, cur, next, cb, HELP ? board + wib : nullptr, refl, idx, j, lane, bytes, cones, evals,
                     vis, no_rx);
  }
  add_stats(tr, cones, vis, bytes, evals, no_rx);
  if constexpr (!HELP) return;
  if (lane == 0) atomicSub(&s_active, 1u);
  // help: take entries of the other warps' slots until no warp of the block runs a
  // cone (a running cone's owner waits for the entries it published, so once
  // s_active reads zero no entry is left).  Bounded: ten seconds at most.
  const long long t0 = clock64();
  unsigned nap = 64;
  for (;;) {
    int v = -1;
    unsigned tk = 0xffffffffu;
    for (int k = 1; k < nw && v < 0; ++k) {
      const int u = wib + k < nw ? wib + k : wib + k - nw;
      tk = help_take(board[u], lane);
      if (tk != 0xffffffffu) v = u;
    }
    if (v >= 0) {
      help_walk(s, tr, next, cb, board[v], tk, lane);
      nap = 64;
      continue;
    }
    bool fin = false;
    if (lane == 0) {
      fin = *(volatile unsigned*)&s_active == 0u;
      if (!fin && clock64() - t0 > wait_cap(tr, 20000000000ll)) {
        atomicExch(tr.err, 4u);
        fin = true;
      }
      if (!fin) __nanosleep(nap);
    }
    if (__shfl_sync(FULL, fin, 0)) break;
    nap = min(nap * 2, 1024u);
  }
}

// All propagation levels in one launch.  A cone of depth d + 1 becomes a task as
// soon as its parent has emitted it, so no level waits for the slowest cone of the
// level before it (each level's last cones otherwise leave most SMs idle).
//   - Per level two ticket counters hand out reflected-cone tasks and Keller-fan
//     tasks (M per diffraction node) in slot order.  A warp takes a ticket with one
//     atomicAdd once the level shows more tasks than tickets; a ticket past the
//     level's current end is held until a parent emits that task, or dropped once
//     the level can grow no more.  (A compare-and-swap claim let only one of the
//     waiting warps succeed per round of the counter's atomic unit: 8-18x slower.)
//   - Per level a count of tasks created and not finished.  Level e can grow no more
//     once the counts of levels 1..e-1, read in that order, are zero: a level-k task
//     is created only by a running level-(k-1) task, and level 1 is complete from
//     the start.  The tree is done when every count reads zero that way.
//   - Per node slot a flag set once its record is written.
// A warp takes the shallowest task available, skipping the levels it has seen final
// with every task ticketed; it leaves once that holds for every level.  Every wait is bounded (ten seconds
// for work, a second and a half for a record): a warp that gives up sets err and
// leaves, and the call reports NIMBUS_ERR_TIMEOUT.  The grid is at most what is
// resident.
struct LevelSet {
  NodeLevel lv[MAX_LEVELS + 1];   // lv[d] for d = 1..max_int; lv[max_int + 1] is the sink
  unsigned long long* take;       // [2 * (MAX_LEVELS + 1)]: tickets handed out per level (reflected, fan)
  uint32_t* err;
  unsigned long long* dbg;        // [20]: where a wait gave up
  int max_int;
};

__device__ __forceinline__ unsigned long long ldv64(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// Tasks level e holds now: reflected cones (kind 0) or fan cones (kind 1).
__device__ __forceinline__ unsigned long long level_total(const LevelSet& L, int e, int kind, int M) {
  const NodeLevel& c = L.lv[e];
  if (kind == 0) return min(*(const volatile uint32_t*)&c.cnt[0], c.cap_r);
  return (unsigned long long)min(*(const volatile uint32_t*)&c.cnt[1], c.cap_d) * (unsigned)M;
}

// Levels 1..e-1 have no task left (read in increasing order), so level e is final.
__device__ __forceinline__ bool levels_done(const LevelSet& L, int e) {
  for (int k = 1; k < e; ++k)
    if (ldv64(L.lv[k].outstanding) != 0ull) return false;
  return true;
}

__global__ void __launch_bounds__(LEVEL_MAX_THREADS, LEVEL_MIN_BLOCKS) k_levels(DScene s, DTrace tr, LevelSet L,
                                                                                 CoarseBuf cb) {
  // each warp walks its own cones' rays (its waiting warps look for cones of any
  // level instead of walking other warps' rays)
  const int lane = threadIdx.x & 31;
  unsigned long long bytes = 0;
  uint32_t cones = 0, vis = 0, evals = 0, no_rx = 0;
  const int M = tr.M;
  int lo = 1;   // lane 0: levels below lo are final and every task of theirs is ticketed
  for (;;) {
    // lane 0 finds a task (level d, kind, ticket t) or learns that the tree is done
    int d = 0, kind = 0;
    unsigned long long t = 0;
    if (lane == 0) {
      const long long t0 = clock64();
      unsigned nap = 128;
      for (;;) {
        int e = lo, k = 0;
        bool held = false;
        for (; e <= L.max_int && !held; ++e)
          for (k = 0; k < 2; ++k)
            if (ldv64(&L.take[2 * e + k]) < level_total(L, e, k, M)) {
              t = atomicAdd(&L.take[2 * e + k], 1ull);
              held = true;
              break;
            }
        if (held) {
          --e;   // the loop's increment ran once more
          // wait for the ticket's task, or drop it once level e is final
          for (;;) {
            if (t < level_total(L, e, k, M)) {
              d = e;
              kind = k;
              break;
            }
            if (levels_done(L, e)) {
              if (t < level_total(L, e, k, M)) {
                d = e;
                kind = k;
              }
              break;
            }
            if (clock64() - t0 > wait_cap(tr, 20000000000ll)) break;
            __nanosleep(nap);
            nap = min(nap * 2, 16384u);
          }
          if (d != 0) break;
          continue;   // dropped: look again
        }
        while (lo <= L.max_int && ldv64(&L.take[2 * lo]) >= level_total(L, lo, 0, M) &&
               ldv64(&L.take[2 * lo + 1]) >= level_total(L, lo, 1, M) && levels_done(L, lo))
          ++lo;
        if (lo > L.max_int) break;   // no level can grow and every task is ticketed: done
        if (clock64() - t0 > wait_cap(tr, 20000000000ll)) {
          if (atomicExch(L.err, 1u) == 0u) {
            L.dbg[0] = 1;
            for (int q = 1; q <= L.max_int && q < 8; ++q) {
              L.dbg[2 * q] = ldv64(&L.take[2 * q]);
              L.dbg[2 * q + 1] = ldv64(L.lv[q].outstanding);
            }
          }
          break;
        }
        // back off while there is nothing to take: the waiting warps' loads of the
        // counters otherwise compete with the working warps' memory traffic
        __nanosleep(nap);
        nap = min(nap * 2, 16384u);
      }
      if (d != 0) {
        // the record of a node made in this launch: wait until it is written
        const uint32_t node = kind == 0 ? (uint32_t)t : (uint32_t)(t / (unsigned)M);
        const uint8_t* rdy = kind == 0 ? L.lv[d].rdy_r : L.lv[d].rdy_d;
        if (rdy) {
          const long long t1 = clock64();
          while (*(const volatile uint8_t*)(rdy + node) == 0) {
            if (clock64() - t1 > wait_cap(tr, 3000000000ll)) {
              if (atomicExch(L.err, 2u) == 0u) {
                L.dbg[0] = 2;
                L.dbg[1] = (unsigned long long)d | ((unsigned long long)kind << 8);
                L.dbg[2] = node;
              }
              d = -1;
              break;
            }
            __nanosleep(32);
          }
          __threadfence();
        }
      }
    }
    d = __shfl_sync(FULL, d, 0);
    if (d <= 0) break;
    kind = __shfl_sync(FULL, kind, 0);
    t = __shfl_sync(FULL, t, 0);
    const uint32_t idx = kind == 0 ? (uint32_t)t : (uint32_t)(t / (unsigned)M);
    const int j = kind == 0 ? 0 : (int)(t % (unsigned)M);
    level_cone<false>(s, tr, L.lv[d], L.lv[d + 1], cb, nullptr, kind == 0, idx, j, lane, bytes, cones, evals, vis,
                      no_rx);
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      atomicAdd(L.lv[d].outstanding, ~0ull);   // this task is finished
    }
  }
  add_stats(tr, cones, vis, bytes, evals, no_rx);
}

// Tasks of the first level (written before the launch) for the single launch.
__global__ void k_levels_init(NodeLevel L1, int M) {
  *L1.outstanding = (unsigned long long)min(L1.cnt[0], L1.cap_r) + (unsigned long long)min(L1.cnt[1], L1.cap_d) * M;
}

// March field of one trace call: the scene's field capped at R+1, lowered to the
// exact L-inf distance around each RX voxel out to radius R.  Exact wherever the
// true distance is <= 1 (so the voxels evaluated are unchanged), a lower bound
// elsewhere (so skipping stays safe).
__global__ void k_march_cap(const uint8_t* in, uint32_t* out, int64_t n, uint32_t cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = min((uint32_t)in[i], cap);
}

__global__ void k_march_rx(DScene s, const int4* rx_vox, int n_rx, uint32_t* m, int R) {
  int side = 2 * R + 1;
  int64_t per = (int64_t)side * side * side;
  int64_t total = per * n_rx;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int j = (int)(i / per);
    int64_t q = i % per;
    int dx = (int)(q % side) - R, dy = (int)((q / side) % side) - R, dz = (int)(q / ((int64_t)side * side)) - R;
    int4 v = rx_vox[j];
    int x = v.x + dx, y = v.y + dy, z = v.z + dz;
    if (!in_grid(s, x, y, z)) continue;
    uint32_t d = (uint32_t)max(abs(dx), max(abs(dy), abs(dz)));
    atomicMin(&m[cell_index(s, x, y, z)], d);
  }
}

__global__ void k_march_pack(const uint32_t* in, uint8_t* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint8_t)min(in[i], 255u);
}

__global__ void k_rx_setup(DScene s, const double* rxd, int n_rx, float4* rx, int4* rx_vox, uint64_t* rx_keys,
                           uint32_t* rx_bits) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_rx) return;
  float p[3] = {(float)rxd[3 * j], (float)rxd[3 * j + 1], (float)rxd[3 * j + 2]};
  const float o[3] = {s.ox, s.oy, s.oz};
  const int dims[3] = {s.nx, s.ny, s.nz};
  int gs[3];
  for (int a = 0; a < 3; ++a) gs[a] = subvoxel_axis(p[a], o[a], s.hs, dims[a] * s.dv - 1);
  int vx = gs[0] / s.dv, vy = gs[1] / s.dv, vz = gs[2] / s.dv;
  long long c = cell_index(s, vx, vy, vz);
  rx[j] = make_float4(p[0], p[1], p[2], 0.f);
  rx_vox[j] = make_int4(vx, vy, vz, 0);
  rx_keys[j] = ((uint64_t)c << 32) | (uint64_t)j;
  atomicOr(&rx_bits[c >> 5], 1u << (c & 31));
}

__global__ void k_tx_setup(const double* txd, int n_tx, float4* tx) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_tx) return;
  tx[j] = make_float4((float)txd[3 * j], (float)txd[3 * j + 1], (float)txd[3 * j + 2], 0.f);
}

// ------------------------------------------------------------------ kappa duplicate limit
struct LevelsView {
  const float4* ra[MAX_LEVELS];
  const float4* rb[MAX_LEVELS];
  const uint32_t* rm[MAX_LEVELS];
  const float4* da[MAX_LEVELS];
  const float4* db[MAX_LEVELS];
  const uint32_t* dm[MAX_LEVELS];
};

// Walk a coarse path's parents: IE, type and label per interaction.
__global__ void k_expand(DScene s, LevelsView L, const uint4* rec, const float* miss, int64_t n, uint32_t* o_tx,
                         uint32_t* o_rx, uint32_t* o_n, uint32_t* o_types, uint32_t* o_ie, uint32_t* o_lab,
                         float* o_miss, uint32_t* o_hash) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint4 r = rec[i];
    uint32_t depth = r.w, ref = r.z, types = 0;
    uint32_t h = 2166136261u;
    for (int q = NB_MAXI - 1; q >= 0; --q) {
      o_ie[i * NB_MAXI + q] = NO_NODE;
      o_lab[i * NB_MAXI + q] = NB_NONE_LABEL;
    }
    for (int q = (int)depth; q >= 1; --q) {
      bool diff = (ref >> 31) != 0;
      uint32_t idx = ref & 0x7fffffffu;
      float4 a = diff ? L.da[q][idx] : L.ra[q][idx];
      float4 b = diff ? L.db[q][idx] : L.rb[q][idx];
      uint32_t m = diff ? L.dm[q][idx] : L.rm[q][idx];
      uint32_t ie = __float_as_uint(a.w);
      o_ie[i * NB_MAXI + q - 1] = ie;
      o_lab[i * NB_MAXI + q - 1] = __float_as_uint(s.ies[ie].rp_lab.w);
      if (diff) types |= 1u << (q - 1);
      ref = __float_as_uint(b.w) | (((m >> 28) & 1u) << 31);
    }
    for (int q = 0; q < (int)depth; ++q) {
      h ^= o_ie[i * NB_MAXI + q];
      h *= 16777619u;
    }
    o_tx[i] = r.x;
    o_rx[i] = r.y;
    o_n[i] = depth;
    o_types[i] = types;
    o_miss[i] = miss[i];
    o_hash[i] = h;
  }
}

__device__ __forceinline__ uint32_t mix32(uint32_t h, uint32_t v) {
  h ^= v + 0x9e3779b9u + (h << 6) + (h >> 2);
  return h;
}

// Group id of (tx, rx, interaction types, labels): open addressing with exact key
// comparison, so distinct label sequences never share a group.
__global__ void k_group(const uint32_t* tx, const uint32_t* rx, const uint32_t* nint, const uint32_t* types,
                        const uint32_t* lab, int64_t n, uint32_t* owner, uint32_t cap_mask, uint32_t* gid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = mix32(mix32(mix32(mix32(0x1234567u, tx[i]), rx[i]), nint[i]), types[i]);
    for (uint32_t q = 0; q < nint[i]; ++q) h = mix32(h, lab[i * NB_MAXI + q]);
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    uint32_t slot = h & cap_mask;
    for (uint32_t probe = 0; probe <= cap_mask; ++probe) {
      uint32_t prev = atomicCAS(&owner[slot], NO_NODE, (uint32_t)i);
      if (prev == NO_NODE) {
        gid[i] = slot;
        break;
      }
      bool same = tx[prev] == tx[i] && rx[prev] == rx[i] && nint[prev] == nint[i] && types[prev] == types[i];
      for (uint32_t q = 0; same && q < nint[i]; ++q) same = lab[prev * NB_MAXI + q] == lab[i * NB_MAXI + q];
      if (same) {
        gid[i] = slot;
        break;
      }
      slot = (slot + 1) & cap_mask;
    }
  }
}

// Sort key: group, then distance of the RX from the cone axis (kappa selection
// reading), then a hash of the IE sequence for ties.
__global__ void k_kappa_keys(const uint32_t* gid, const float* miss, const uint32_t* hash, int64_t n, uint64_t* keys,
                             uint32_t* vals) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t mb = __float_as_uint(fmaxf(miss[i], 0.f)) & 0x7fffffffu;
    keys[i] = ((uint64_t)gid[i] << 39) | ((uint64_t)mb << 8) | (uint64_t)(hash[i] & 0xffu);
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_kappa_keep(const uint64_t* keys, int64_t n, int kappa, uint32_t* keep) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t g = keys[i] >> 39;
    int64_t lo = 0, hi = i;
    while (lo < hi) {  // first position of this group
      int64_t mid = (lo + hi) >> 1;
      if ((keys[mid] >> 39) < g) lo = mid + 1;
      else hi = mid;
    }
    keep[i] = (i - lo) < kappa ? 1u : 0u;
  }
}

__global__ void k_kappa_compact(const uint32_t* keep, const uint32_t* pos, const uint32_t* order, int64_t n,
                                const uint32_t* tx, const uint32_t* rx, const uint32_t* nint, const uint32_t* types,
                                const uint32_t* ie, const uint32_t* lab, const float* miss, const uint32_t* gid,
                                CoarseObj out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    uint32_t src = order[i];
    uint32_t d = pos[i];
    out.tx[d] = tx[src];
    out.rx[d] = rx[src];
    out.nint[d] = nint[src];
    out.types[d] = types[src];
    out.miss[d] = miss[src];
    out.gid[d] = gid[src];
    for (int q = 0; q < NB_MAXI; ++q) {
      out.ie[(size_t)d * NB_MAXI + q] = ie[(size_t)src * NB_MAXI + q];
      out.lab[(size_t)d * NB_MAXI + q] = lab[(size_t)src * NB_MAXI + q];
    }
  }
}

unsigned persistent_grid(int block) {
  static int sms = 0;
  if (!sms) sms = num_sms();
  return (unsigned)(sms * (2048 / block));
}

}  // namespace

int trace_coarse(Mem& mem, SceneObj* S, const double* txh, int n_tx, const double* rxh, int n_rx,
                 const nimbus_trace_params* p, CoarseObj* C, cudaStream_t st, const Tuning& tn) {
  std::string* err = mem.err;
  if (n_tx < 1 || n_rx < 0 || !txh || (n_rx > 0 && !rxh) || n_tx > 65535) {
    *err = "trace: invalid TX/RX arrays";
    return NIMBUS_ERR_ARG;
  }
  if (p->max_refl < 0 || p->max_diff < 0 || p->kappa < 1 || !(p->cone_half_angle > 0) ||
      !(p->cone_half_angle < 1.5) || !(p->launch_spacing > 0) || p->launch_mode < 0 || p->launch_mode > 1) {
    *err = "trace: invalid parameters";
    return NIMBUS_ERR_ARG;
  }
  const int max_int = p->max_int >= 0 ? p->max_int : p->max_refl + p->max_diff;
  if (max_int > NB_MAXI || p->max_refl > 15 || p->max_diff > 15) {
    *err = "trace: too many interactions";
    return NIMBUS_ERR_ARG;
  }
  const DScene& s = S->d;
  const long long launches0 = g_launches.load();
  C->mem = &mem;
  C->max_refl = std::min(p->max_refl, max_int);
  C->n_tx = n_tx;
  C->n_rx = n_rx;
  // TX/RX on the host for the grid check, on the device for the kernels
  std::vector<double> th(3 * n_tx), rh(3 * (size_t)n_rx);
  NB_CUDA(err, cudaMemcpy(th.data(), txh, th.size() * sizeof(double), cudaMemcpyDefault));
  if (n_rx) NB_CUDA(err, cudaMemcpy(rh.data(), rxh, rh.size() * sizeof(double), cudaMemcpyDefault));
  for (int i = 0; i < n_tx + n_rx; ++i) {
    const double* q = i < n_tx ? &th[3 * i] : &rh[3 * (i - n_tx)];
    for (int a = 0; a < 3; ++a) {
      double rel = (q[a] - S->origin[a]) / S->params.voxel_size;
      if (!(rel >= 0.0 && rel < (double)S->dims[a])) {
        *err = "trace: a TX or RX lies outside the voxel grid";
        return NIMBUS_ERR_ARG;
      }
    }
  }
  NB_TRY(C->own(&C->txd, 3 * n_tx, st));
  NB_TRY(C->own(&C->rxd, std::max(1, 3 * n_rx), st));
  NB_CUDA(err, cudaMemcpyAsync(C->txd, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (n_rx) NB_CUDA(err, cudaMemcpyAsync(C->rxd, rh.data(), rh.size() * sizeof(double), cudaMemcpyHostToDevice, st));

  Scratch sc(&mem, st);
  const int64_t n_cells = s.n_cells;
  const int64_t n_ie = s.n_ie;
  DTrace tr;
  std::memset(&tr, 0, sizeof tr);
  const double alpha = p->cone_half_angle;
  const double alpha0 = std::max(alpha, p->launch_spacing / std::sqrt(2.0));
  tr.sin_a = (float)std::sin(alpha);
  tr.cos_a = (float)std::cos(alpha);
  tr.sin_a0 = (float)std::sin(alpha0);
  tr.cos_a0 = (float)std::cos(alpha0);
  tr.M = (int)std::ceil(PI_D / alpha);
  tr.dphi = (float)(2.0 * PI_D / tr.M);
  tr.sep_eps = (float)p->sep_eps;
  tr.max_refl = p->max_refl;
  tr.max_diff = p->max_diff;
  tr.max_int = max_int;
  tr.n_launch = p->n_launch > 0 ? p->n_launch
                                : (int)std::llround(4.0 * PI_D / (p->launch_spacing * p->launch_spacing));
  tr.n_tx = n_tx;
  tr.n_rx = n_rx;
  tr.n_ie = (uint32_t)n_ie;
  tr.n_edges = (uint32_t)s.n_edges;
  tr.golden = PI_D * (3.0 - std::sqrt(5.0));
  tr.ie_words = (int)((n_ie + 31) / 32);
  float4 *tx4, *rx4;
  int4* rx_vox;
  uint64_t *rx_keys, *rx_keys_alt;
  uint32_t *rx_vals, *rx_vals_alt, *rx_bits, *mtmp, *vis_ie, *vis_rx, *first_bits, *los, *overflow;
  uint8_t* march;
  unsigned long long* stats;
  NB_TRY(sc.get(&tx4, n_tx));
  NB_TRY(sc.get(&rx4, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_vox, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_keys, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_keys_alt, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_vals, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_vals_alt, std::max(1, n_rx)));
  NB_TRY(sc.get(&rx_bits, (n_cells + 31) / 32));
  NB_TRY(sc.get(&mtmp, n_cells));
  NB_TRY(sc.get(&march, n_cells));
  NB_TRY(sc.get(&vis_ie, std::max<int64_t>(1, (int64_t)n_tx * tr.ie_words)));
  NB_TRY(sc.get(&vis_rx, std::max<int64_t>(1, (int64_t)n_tx * n_rx)));
  NB_TRY(sc.get(&first_bits, std::max<int64_t>(1, (int64_t)n_tx * tr.ie_words)));
  NB_TRY(sc.get(&los, std::max<int64_t>(1, (int64_t)n_tx * n_rx)));
  NB_TRY(sc.get(&overflow, 2));
  NB_TRY(sc.get(&stats, N_STATS * N_STAGES));
  const int R = 8;
  tr.tx = tx4;
  tr.rx = rx4;
  tr.march = march;
  tr.rx_bits = rx_bits;
  tr.rx_sorted = rx_keys;
  tr.n_rx_sorted = n_rx;
  tr.vis_ie = vis_ie;
  tr.vis_rx = vis_rx;
  tr.stats = stats;
  tr.overflow = overflow;
  // optional per-RX owner TX and interaction limit (request batching); each TX's
  // tree is then expanded only as deep as the deepest RX it serves
  tr.rx_owner = nullptr;
  tr.rx_max_int = nullptr;
  tr.tx_max_int = nullptr;
  if (n_rx > 0 && (p->rx_owner || p->rx_max_int)) {
    std::vector<int32_t> own(n_rx, -1), mx(n_rx, -1), lim(n_tx, 0);
    if (p->rx_owner) NB_CUDA(err, cudaMemcpy(own.data(), p->rx_owner, n_rx * sizeof(int32_t), cudaMemcpyDefault));
    if (p->rx_max_int) NB_CUDA(err, cudaMemcpy(mx.data(), p->rx_max_int, n_rx * sizeof(int32_t), cudaMemcpyDefault));
    for (int j = 0; j < n_rx; ++j) {
      if (own[j] >= n_tx) {
        *err = "trace: rx_owner names a TX that does not exist";
        return NIMBUS_ERR_ARG;
      }
      int d = mx[j] >= 0 ? std::min(mx[j], max_int) : max_int;
      if (own[j] >= 0) lim[own[j]] = std::max(lim[own[j]], d);
      else
        for (int t = 0; t < n_tx; ++t) lim[t] = std::max(lim[t], d);
    }
    int32_t *d_own, *d_mx, *d_lim;
    NB_TRY(sc.get(&d_own, n_rx));
    NB_TRY(sc.get(&d_mx, n_rx));
    NB_TRY(sc.get(&d_lim, n_tx));
    NB_CUDA(err, cudaMemcpyAsync(d_own, own.data(), n_rx * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_mx, mx.data(), n_rx * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NB_CUDA(err, cudaMemcpyAsync(d_lim, lim.data(), n_tx * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    tr.rx_owner = d_own;
    tr.rx_max_int = d_mx;
    tr.tx_max_int = d_lim;
  }

  // bounded buffers: nodes per level and coarse paths
  const int64_t cap_nodes = p->max_nodes > 0 ? p->max_nodes : (int64_t)8 << 20;
  const int64_t cap_coarse = p->max_coarse > 0 ? p->max_coarse : (int64_t)8 << 20;
  if (cap_nodes >= (1ll << 31) || cap_coarse >= (1ll << 31)) {
    *err = "trace: buffer bounds too large";
    return NIMBUS_ERR_ARG;
  }
  NodeLevel lv[MAX_LEVELS];
  std::memset(lv, 0, sizeof lv);
  uint32_t* cnts;
  NB_TRY(sc.get(&cnts, 2 * MAX_LEVELS));
  for (int d = 1; d <= max_int; ++d) {
    NodeLevel& L = lv[d];
    L.cap_r = (uint32_t)cap_nodes;
    L.cap_d = (uint32_t)std::max<int64_t>(1024, cap_nodes / 8);
    if (p->max_diff == 0) L.cap_d = 1;
    if (p->max_refl == 0) L.cap_r = 1;
    NB_TRY(sc.get(&L.ra, L.cap_r));
    NB_TRY(sc.get(&L.rb, L.cap_r));
    NB_TRY(sc.get(&L.rm, L.cap_r));
    NB_TRY(sc.get(&L.da, L.cap_d));
    NB_TRY(sc.get(&L.db, L.cap_d));
    NB_TRY(sc.get(&L.dm, L.cap_d));
    L.cnt = cnts + 2 * d;
  }
  CoarseBuf cb;
  cb.cap = (uint32_t)cap_coarse;
  NB_TRY(sc.get(&cb.rec, cb.cap));
  NB_TRY(sc.get(&cb.miss, cb.cap));
  cb.cnt = cnts;  // slot 0 of level 0 counts the coarse paths
  const int64_t nflag = (int64_t)n_tx * n_ie;
  uint32_t *fr = nullptr, *fd = nullptr, *pr = nullptr, *pd = nullptr, *tot = nullptr;
  if (max_int >= 1) {
    NB_TRY(sc.get(&fr, std::max<int64_t>(1, nflag)));
    NB_TRY(sc.get(&fd, std::max<int64_t>(1, nflag)));
    NB_TRY(sc.get(&pr, std::max<int64_t>(1, nflag)));
    NB_TRY(sc.get(&pd, std::max<int64_t>(1, nflag)));
    NB_TRY(sc.get(&tot, 2));
  }
  unsigned long long* task_ctr;   // cones handed out so far, one counter per level
  NB_TRY(sc.get(&task_ctr, MAX_LEVELS));
  // single-launch propagation: task counters, created-not-finished count, error flag
  // and per-slot ready flags of the levels made inside the launch
  const bool queue = tn.level_queue != 0 && max_int >= 1;
  LevelSet LS;
  std::memset(&LS, 0, sizeof LS);
  unsigned long long* q_ctr = nullptr;
  uint32_t* q_err = nullptr;
  size_t rdy_bytes = 0;
  uint8_t* rdy = nullptr;
  NB_TRY(sc.get(&q_err, 4));   // both layouts: a bounded wait gave up, or a self-check failed
  tr.err = q_err;
  if (queue) {
    NB_TRY(sc.get(&q_ctr, 2 * (MAX_LEVELS + 1) + 1 + 20 + MAX_LEVELS + 1));
    for (int d = 2; d <= max_int; ++d) rdy_bytes += (size_t)lv[d].cap_r + lv[d].cap_d;
    NB_TRY(sc.get(&rdy, std::max<size_t>(1, rdy_bytes)));
    size_t off = 0;
    for (int d = 1; d <= max_int; ++d) {
      lv[d].outstanding = q_ctr + 2 * (MAX_LEVELS + 1) + 1 + 20 + d;
      if (d >= 2) {
        lv[d].rdy_r = rdy + off;
        off += lv[d].cap_r;
        lv[d].rdy_d = rdy + off;
        off += lv[d].cap_d;
      }
      LS.lv[d] = lv[d];
    }
    NodeLevel sink;
    std::memset(&sink, 0, sizeof sink);
    sink.cnt = cnts + 2 * MAX_LEVELS - 2;
    LS.lv[max_int + 1] = sink;
    LS.take = q_ctr;
    LS.dbg = q_ctr + 2 * (MAX_LEVELS + 1) + 1;
    LS.err = q_err;
    LS.max_int = max_int;
  }
  // the sorts and scans of the stretch below draw from this arena
  const size_t arena_bytes =
      radix_arena_bytes(n_rx, 64) + (max_int >= 1 ? 2 * scan_arena_bytes(nflag, true) : 0);
  char* arena;
  NB_TRY(sc.get(&arena, std::max<size_t>(1, arena_bytes)));
  const unsigned PG = persistent_grid(256);
  // the levels' grids are what is resident (the single launch's warps wait for one
  // another's work, and a block of the per-depth launch helps only its own warps)
  const bool help = tn.level_help != 0;
  const size_t board_bytes = help ? (size_t)(tn.level_block / 32) * sizeof(HelpSlot) : 0;
  auto* k_lev = help ? k_level<true> : k_level<false>;
  int l_blocks = 0, q_blocks = 0;
  NB_CUDA(err, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l_blocks, k_lev, tn.level_block, board_bytes));
  if (queue) NB_CUDA(err, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q_blocks, k_levels, tn.level_block, 0));
  const unsigned LG = (unsigned)(num_sms() * std::max(1, l_blocks));
  const unsigned QG = (unsigned)(num_sms() * std::max(1, q_blocks));
  StageTimer tm(st);
  const int e0 = stretch_event(tm, mem, GRAPH_TRACE, 0), e1 = stretch_event(tm, mem, GRAPH_TRACE, 1),
            e2 = stretch_event(tm, mem, GRAPH_TRACE, 2), e3 = stretch_event(tm, mem, GRAPH_TRACE, 3),
            e4 = stretch_event(tm, mem, GRAPH_TRACE, 4);
  DTrace tr_vis = tr, tr_pri = tr, tr_lev = tr;
  tr_vis.stats = stats + STAGE_VIS * N_STATS;
  tr_pri.stats = stats + STAGE_PRIMARY * N_STATS;
  tr_lev.stats = stats + STAGE_LEVELS * N_STATS;
  tr_lev.err = q_err;
  tr_lev.wait_limit = tn.wait_limit;
  tr_lev.rx_first = tn.level_rx_first;

  // From the RX table to the last depth nothing returns to the host: the march field,
  // the transmission phase and every propagation level over all TX/RX pairs form one
  // stretch, issued as one CUDA graph by default.
  NB_TRY(run_stretch(mem, st, tn.graph != 0, GRAPH_TRACE, [&](cudaStream_t q) -> int {
    Scratch ws(&mem, q);
    ws.arena = arena;
    ws.arena_cap = arena_bytes;
    NB_CUDA(err, cudaMemsetAsync(rx_bits, 0, ((n_cells + 31) / 32) * sizeof(uint32_t), q));
    NB_CUDA(err, cudaMemsetAsync(vis_ie, 0, std::max<int64_t>(1, (int64_t)n_tx * tr.ie_words) * 4, q));
    NB_CUDA(err, cudaMemsetAsync(first_bits, 0, std::max<int64_t>(1, (int64_t)n_tx * tr.ie_words) * 4, q));
    NB_CUDA(err, cudaMemsetAsync(los, 0xff, std::max<int64_t>(1, (int64_t)n_tx * n_rx) * 4, q));
    NB_CUDA(err, cudaMemsetAsync(overflow, 0, 2 * sizeof(uint32_t), q));
    NB_CUDA(err, cudaMemsetAsync(stats, 0, N_STATS * N_STAGES * sizeof(unsigned long long), q));
    NB_CUDA(err, cudaMemsetAsync(cnts, 0, 2 * MAX_LEVELS * sizeof(uint32_t), q));
    NB_CUDA(err, cudaMemsetAsync(task_ctr, 0, MAX_LEVELS * sizeof(unsigned long long), q));
    k_tx_setup<<<grid_for(n_tx, 64), 64, 0, q>>>(C->txd, n_tx, tx4);
    NB_LAUNCHED(err);
    if (n_rx > 0) {
      k_rx_setup<<<grid_for(n_rx, 64), 64, 0, q>>>(s, C->rxd, n_rx, rx4, rx_vox, rx_keys, rx_bits);
      NB_LAUNCHED(err);
      NB_CUDA(err, cudaMemsetAsync(rx_vals, 0, n_rx * sizeof(uint32_t), q));
      NB_TRY(radix_sort(ws, rx_keys, rx_vals, rx_keys_alt, rx_vals_alt, n_rx, 64));
    }
    k_march_cap<<<std::min<unsigned>(grid_for(n_cells, 256), 2048u), 256, 0, q>>>(s.march, mtmp, n_cells, R + 1);
    NB_LAUNCHED(err);
    if (n_rx > 0) {
      int64_t work = (int64_t)(2 * R + 1) * (2 * R + 1) * (2 * R + 1) * n_rx;
      k_march_rx<<<std::min<unsigned>(grid_for(work, 256), 4096u), 256, 0, q>>>(s, rx_vox, n_rx, mtmp, R);
      NB_LAUNCHED(err);
    }
    k_march_pack<<<std::min<unsigned>(grid_for(n_cells, 256), 2048u), 256, 0, q>>>(mtmp, march, n_cells);
    NB_LAUNCHED(err);
    // transmission phase
    tm.record(e0, q);
    k_vis_tables<<<PG, 256, 0, q>>>(s, tr_vis);
    NB_LAUNCHED(err);
    tm.record(e1, q);
    if (p->launch_mode == 1) {
      // the paper's launch: a ray toward every IE and RX, i.e. the visibility tables
      NB_CUDA(err, cudaMemcpyAsync(first_bits, vis_ie, std::max<int64_t>(1, (int64_t)n_tx * tr.ie_words) * 4,
                                   cudaMemcpyDeviceToDevice, q));
      if ((int64_t)n_tx * n_rx > 0) {
        k_los_from_vis<<<grid_for((int64_t)n_tx * n_rx, 128), 128, 0, q>>>(tr, los);
        NB_LAUNCHED(err);
      }
    } else {
      k_primary<<<PG, 256, 0, q>>>(s, tr_pri, first_bits, los);
      NB_LAUNCHED(err);
    }
    tm.record(e2, q);
    k_los<<<grid_for((int64_t)n_tx * n_rx, 128), 128, 0, q>>>(tr, los, cb);
    NB_LAUNCHED(err);
    if (max_int >= 1) {
      if (nflag > 0) {
        k_first_flags<<<PG, 256, 0, q>>>(s, tr, first_bits, fr, fd);
        NB_LAUNCHED(err);
      }
      NB_TRY(exclusive_scan(ws, fr, pr, nflag, tot));
      NB_TRY(exclusive_scan(ws, fd, pd, nflag, tot + 1));
      if (nflag > 0) {
        k_first_nodes<<<PG, 256, 0, q>>>(s, tr, fr, pr, fd, pd, lv[1]);
        NB_LAUNCHED(err);
      }
      k_first_counts<<<1, 1, 0, q>>>(tot, tot + 1, lv[1]);
      NB_LAUNCHED(err);
    }
    // propagation phase: one launch per depth, or one launch for all depths
    NB_CUDA(err, cudaMemsetAsync(q_err, 0, 4 * sizeof(uint32_t), q));
    if (queue) {
      NB_CUDA(err, cudaMemsetAsync(q_ctr, 0, (2 * (MAX_LEVELS + 1) + 1 + 20 + MAX_LEVELS + 1) * sizeof(unsigned long long), q));
      if (rdy_bytes) NB_CUDA(err, cudaMemsetAsync(rdy, 0, rdy_bytes, q));
      k_levels_init<<<1, 1, 0, q>>>(lv[1], tr.M);
      NB_LAUNCHED(err);
    }
    tm.record(e3, q);
    if (queue) {
      k_levels<<<QG, tn.level_block, 0, q>>>(s, tr_lev, LS, cb);
      NB_LAUNCHED(err);
    } else {
      for (int d = 1; d <= max_int; ++d) {
        NodeLevel next = d < max_int ? lv[d + 1] : lv[0];
        if (d == max_int) {
          next.cap_r = 0;
          next.cap_d = 0;
          next.cnt = cnts + 2 * MAX_LEVELS - 2;  // unused sink
        }
        k_lev<<<LG, tn.level_block, board_bytes, q>>>(s, tr_lev, lv[d], next, cb, task_ctr + d);
        NB_LAUNCHED(err);
      }
    }
    tm.record(e4, q);
    return NIMBUS_OK;
  }));
  // read the sizes back
  uint32_t hc[2 * MAX_LEVELS], hov[2];
  unsigned long long hs[N_STATS * N_STAGES];
  NB_CUDA(err, cudaMemcpyAsync(hc, cnts, sizeof hc, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaMemcpyAsync(hov, overflow, sizeof hov, cudaMemcpyDeviceToHost, st));
  NB_CUDA(err, cudaMemcpyAsync(hs, stats, sizeof hs, cudaMemcpyDeviceToHost, st));
  uint32_t hq[4] = {0, 0, 0, 0};
  NB_CUDA(err, cudaMemcpyAsync(hq, q_err, sizeof hq, cudaMemcpyDeviceToHost, st));
  const uint32_t hqerr = hq[0];
  NB_CUDA(err, cudaStreamSynchronize(st));
  if (hqerr == 3u || hqerr == 4u) {
    *err = hqerr == 3u ? "trace: a cone's wait for the visibility rays other warps took gave up"
                       : "trace: a warp's wait for the cones of its block gave up";
    return NIMBUS_ERR_TIMEOUT;
  }
  if (hqerr >= 5u) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "trace: propagation self-check %u failed (%u %u %u); the access was skipped",
                  hqerr, hq[1], hq[2], hq[3]);
    *err = buf;
    return NIMBUS_ERR_STATE;
  }
  if (hqerr) {
    unsigned long long hd[20];
    cudaMemcpy(hd, LS.dbg, sizeof hd, cudaMemcpyDeviceToHost);
    char buf[512];
    int o = std::snprintf(buf, sizeof buf, "trace: a wait of the single-launch propagation gave up (%llu: %llu %llu |",
                          hd[0], hd[1], hd[2]);
    for (int d = 1; d <= max_int && d < 8 && o < 400; ++d)
      o += std::snprintf(buf + o, sizeof buf - o, " L%d tickets %llu open %llu nodes %u/%u", d, hd[2 * d],
                         hd[2 * d + 1], hc[2 * d], hc[2 * d + 1]);
    *err = std::string(buf) + ")";
    return NIMBUS_ERR_TIMEOUT;
  }
  nimbus_path_counts& cnt = C->counts;
  std::memset(&cnt, 0, sizeof cnt);
  const int64_t n_raw = std::min<int64_t>(hc[0], cb.cap);
  cnt.n_coarse_raw = hc[0];
  for (int g = 0; g < N_STAGES; ++g) {
    cnt.n_cones += (int64_t)hs[g * N_STATS + ST_CONES];
    cnt.n_vis += (int64_t)hs[g * N_STATS + ST_VIS];
    cnt.bytes_read += (int64_t)hs[g * N_STATS + ST_BYTES];
  }
  cnt.bytes_primary = (int64_t)hs[STAGE_PRIMARY * N_STATS + ST_BYTES];
  cnt.bytes_levels = (int64_t)hs[STAGE_LEVELS * N_STATS + ST_BYTES];
  cnt.n_cones_no_rx = (int64_t)hs[STAGE_LEVELS * N_STATS + ST_NO_RX];
  cnt.n_levels = max_int;
  cnt.ms_vis = tm.ms(e0, e1);
  cnt.ms_primary = tm.ms(e1, e2);
  cnt.ms_levels = tm.ms(e3, e4);
  for (int d = 1; d <= max_int; ++d) cnt.n_nodes += (int64_t)hc[2 * d] + hc[2 * d + 1];
  cnt.needed_nodes = hov[0];
  cnt.needed_coarse = hov[1];
  cnt.overflow = (hov[0] != 0 || hov[1] != 0) ? 1 : 0;

  // kappa: group, rank by miss, keep at most kappa per group
  C->n = 0;
  const int e5 = tm.mark();
  int e6 = e5;
  if (n_raw > 0) {
    uint32_t *e_tx, *e_rx, *e_n, *e_types, *e_ie, *e_lab, *e_hash, *gid, *owner, *keep, *pos, *vals, *vals_alt,
        *n_keep;
    float* e_miss;
    uint64_t *keys, *keys_alt;
    NB_TRY(sc.get(&e_tx, n_raw));
    NB_TRY(sc.get(&e_rx, n_raw));
    NB_TRY(sc.get(&e_n, n_raw));
    NB_TRY(sc.get(&e_types, n_raw));
    NB_TRY(sc.get(&e_ie, n_raw * NB_MAXI));
    NB_TRY(sc.get(&e_lab, n_raw * NB_MAXI));
    NB_TRY(sc.get(&e_hash, n_raw));
    NB_TRY(sc.get(&e_miss, n_raw));
    NB_TRY(sc.get(&gid, n_raw));
    uint32_t cap_h = 1024;
    while ((int64_t)cap_h < 2 * n_raw) cap_h <<= 1;
    if (cap_h > (1u << 25)) {
      *err = "trace: too many coarse paths for the kappa step";
      return NIMBUS_ERR_OVERFLOW;
    }
    NB_TRY(sc.get(&owner, cap_h));
    NB_CUDA(err, cudaMemsetAsync(owner, 0xff, cap_h * sizeof(uint32_t), st));
    LevelsView LV;
    std::memset(&LV, 0, sizeof LV);
    for (int d = 1; d <= max_int; ++d) {
      LV.ra[d] = lv[d].ra; LV.rb[d] = lv[d].rb; LV.rm[d] = lv[d].rm;
      LV.da[d] = lv[d].da; LV.db[d] = lv[d].db; LV.dm[d] = lv[d].dm;
    }
    const unsigned G = std::min<unsigned>(grid_for(n_raw, 256), PG);
    k_expand<<<G, 256, 0, st>>>(s, LV, cb.rec, cb.miss, n_raw, e_tx, e_rx, e_n, e_types, e_ie, e_lab, e_miss, e_hash);
    NB_LAUNCHED(err);
    k_group<<<G, 256, 0, st>>>(e_tx, e_rx, e_n, e_types, e_lab, n_raw, owner, cap_h - 1, gid);
    NB_LAUNCHED(err);
    NB_TRY(sc.get(&keys, n_raw));
    NB_TRY(sc.get(&keys_alt, n_raw));
    NB_TRY(sc.get(&vals, n_raw));
    NB_TRY(sc.get(&vals_alt, n_raw));
    NB_TRY(sc.get(&keep, n_raw));
    NB_TRY(sc.get(&pos, n_raw));
    NB_TRY(sc.get(&n_keep, 1));
    k_kappa_keys<<<G, 256, 0, st>>>(gid, e_miss, e_hash, n_raw, keys, vals);
    NB_LAUNCHED(err);
    int gbits = bits_for(cap_h - 1);
    NB_TRY(radix_sort(sc, keys, vals, keys_alt, vals_alt, n_raw, 39 + gbits));
    k_kappa_keep<<<G, 256, 0, st>>>(keys, n_raw, p->kappa, keep);
    NB_LAUNCHED(err);
    NB_TRY(exclusive_scan(sc, keep, pos, n_raw, n_keep));
    uint32_t hk = 0;
    NB_CUDA(err, cudaMemcpyAsync(&hk, n_keep, sizeof hk, cudaMemcpyDeviceToHost, st));
    NB_CUDA(err, cudaStreamSynchronize(st));
    C->n = hk;
    C->n_groups_cap = cap_h;
    NB_TRY(C->own(&C->tx, std::max<int64_t>(1, hk), st));
    NB_TRY(C->own(&C->rx, std::max<int64_t>(1, hk), st));
    NB_TRY(C->own(&C->nint, std::max<int64_t>(1, hk), st));
    NB_TRY(C->own(&C->types, std::max<int64_t>(1, hk), st));
    NB_TRY(C->own(&C->ie, std::max<int64_t>(1, hk) * NB_MAXI, st));
    NB_TRY(C->own(&C->lab, std::max<int64_t>(1, hk) * NB_MAXI, st));
    NB_TRY(C->own(&C->miss, std::max<int64_t>(1, hk), st));
    NB_TRY(C->own(&C->gid, std::max<int64_t>(1, hk), st));
    k_kappa_compact<<<G, 256, 0, st>>>(keep, pos, vals, n_raw, e_tx, e_rx, e_n, e_types, e_ie, e_lab, e_miss, gid,
                                       *C);
    NB_LAUNCHED(err);
    e6 = tm.mark();
  }
  cnt.n_coarse = C->n;
  NB_CUDA(err, cudaStreamSynchronize(st));
  cnt.ms_kappa = tm.ms(e5, e6);
  cnt.launches = g_launches.load() - launches0;
  if (cnt.overflow) {
    *err = "trace: a bounded buffer overflowed (see needed_nodes / needed_coarse)";
    return NIMBUS_ERR_OVERFLOW;
  }
  return NIMBUS_OK;
}

}  // namespace nb
