// FP64 CPU oracle for the point-cloud ray launcher of
// "A Ray Launching Approach for Computing Exact Paths with Point Clouds"
// (Vaara, Sangi, Bordallo Lopez, Heikkila; arXiv 2402.13747).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
// CPU-baseline / reference leg load this library.  It shares no code, header,
// table or constant generator with the CUDA library, and neither includes the
// other.
//
// Plain, slow, single-threaded, FP64.  The three components of Section 2 run in
// the paper's order: voxelisation (Section 2.1), coarse path tracing
// (Section 2.2: transmission, propagation, voxel cone tracing, Eq. 1
// intersections) and path refinement (Section 2.3: Eq. 2 minimised by gradient
// descent, visibility, label and first-Fresnel-zone duplicate removal).
// Where the paper is silent the reading used is stated next to the code.
// Pins (tests/test_oracle_pins.py) fix voxelisation, the march field, Eq. 1,
// visibility, the cone test and the refined exact paths (image method, Keller point,
// a reflection and a diffraction in either order) against closed forms and brute
// force; tests/test_oracle_mutants.py checks that planted mistakes fail them.  The
// secant placement after a sign change of f is pinned on two sheets whose Eq. 1
// surface has a closed form (both marches; also the re-projection of a target that
// lies on the surface), the final visibility check on a path
// that passes just outside a panel, and the RX reception sphere on a single launch
// cone.  The coarse-path set and the kappa choice on noisy clouds have no
// closed form: parity unpinned beyond their invariants (kappa, depth limits) and the
// exact paths they refine to.
// The only FP32 arithmetic is the subvoxel binning, which both sides perform with
// the same correctly rounded FP32 operations so that the point-to-subvoxel
// assignment is bit-identical (binning reading).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <set>
#include <tuple>
#include <vector>

extern "C" {
// Parameters: same meaning as the library's parameter block, declared here on
// its own (the oracle includes nothing from the library).
typedef struct {
  double voxel_size;       // h: low-resolution voxel edge [m] (Table 1)
  double cone_half_angle;  // alpha [rad], constant for all cones (Section 2.2.4)
  double launch_spacing;   // Delta [rad] of the uniform TX launch
  double sdf_sigma;        // Gaussian width of the Eq. 1 weights [m]
  double sdf_eps;          // |f| "near zero" threshold [m] (Section 2.2.1)
  double vis_ignore;       // self-hit ignore distance near path nodes [m]
  double sep_eps;          // reflection separation plane offset [m]
  double delta;            // convergence threshold (Table 1)
  double gamma;            // gradient-descent step scale
  double grad_stop;        // stop once ||grad|| < grad_stop
  double freq_hz;          // carrier frequency (Table 1)
  int32_t dv;              // voxel division factor D_v (Table 1)
  int32_t max_refl;
  int32_t max_diff;
  int32_t max_int;         // maximum number of interactions (Table 1)
  int32_t kappa;           // coarse path duplicate limit (Table 1)
  int32_t n_launch;        // number of uniform launch directions
  int32_t sdf_max_steps;
  int32_t rho;             // refinement iterations (Table 1)
  int32_t launch_mode;     // 0: uniform launch; 1: a ray toward every IE and RX (Section 2.2.2)
} oracle_params;
}

namespace {

constexpr uint32_t NONE_LABEL = 0xFFFFFFFFu;
constexpr int MAXI = 8;                      // interactions per path, upper bound
constexpr double C_LIGHT = 299792458.0;
constexpr double PI = 3.14159265358979323846;

// --------------------------------------------------------------------------- vectors
struct V3 {
  double x = 0, y = 0, z = 0;
};
inline V3 mk(double x, double y, double z) { V3 v; v.x = x; v.y = y; v.z = z; return v; }
inline V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator*(double s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { double n = norm(a); return n > 0 ? (1.0 / n) * a : a; }
inline double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// Orthonormal basis (u, v) completing the unit vector n: the branchless
// construction of Duff et al., "Building an Orthonormal Basis, Revisited" (2017).
void onb(V3 n, V3* u, V3* v) {
  double sign = std::copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *u = mk(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *v = mk(b, sign + n.y * n.y * a, -n.y);
}

// --------------------------------------------------------------------------- scene
enum { IE_POINT = 0, IE_EDGE = 1 };
enum { T_REFL = 0, T_DIFF = 1 };

struct Edge {
  V3 p0, p1, n0, n1;
  uint32_t label;
};

// Intersectable entity (Section 2.1): a subvoxel's points of one label, or a
// diffraction edge segment inside a subvoxel.  Each has a label and a ray
// reception point.  RX entities are added per trace call (TraceCtx).
struct IE {
  int kind = IE_POINT;
  uint32_t label = 0;
  uint8_t material = 0;
  int64_t cell = 0;          // low-resolution voxel (linear index)
  int gs[3] = {0, 0, 0};     // global subvoxel coordinates
  V3 rp;                     // ray reception point
  V3 normal;                 // point IE: normalised mean normal
  V3 bbc;                    // point IE: centre of the points' bounding box
  V3 sc;                     // subvoxel centre (bounding sphere centre)
  int64_t p_begin = 0, p_count = 0;
  int edge = -1;             // edge IE: edge index and parameter range on it
  double t0 = 0, t1 = 0;
};

struct Scene {
  oracle_params p;
  double h = 0, hs = 0, r_vox = 0, r_sub = 0;
  V3 origin;
  int dims[3] = {0, 0, 0};
  int64_t n_cells = 0;
  float o32[3] = {0, 0, 0};
  float hs32 = 0;
  std::vector<V3> pts, nrm;           // point positions/normals grouped by IE
  std::vector<IE> ies;                // sorted by (voxel, subvoxel, kind, label|edge)
  std::vector<int64_t> cell_begin;    // first IE of each voxel
  std::vector<int32_t> cell_count;    // number of IEs in each voxel
  std::vector<int32_t> march;         // L-infinity distance to the nearest voxel with IEs
  std::vector<Edge> edges;
};

inline int64_t cell_of(const Scene& s, int vx, int vy, int vz) {
  return ((int64_t)vz * s.dims[1] + vy) * s.dims[0] + vx;
}
inline bool in_grid(const Scene& s, int vx, int vy, int vz) {
  return vx >= 0 && vy >= 0 && vz >= 0 && vx < s.dims[0] && vy < s.dims[1] && vz < s.dims[2];
}
inline V3 voxel_center(const Scene& s, int vx, int vy, int vz) {
  return mk(s.origin.x + (vx + 0.5) * s.h, s.origin.y + (vy + 0.5) * s.h, s.origin.z + (vz + 0.5) * s.h);
}

// Subvoxel of a position (Section 2.1).  Binning reading: the same FP32 op
// sequence on both sides -- (x - o) then / h_s, each correctly rounded, then
// floor -- so points on subvoxel faces fall on the same side everywhere.
void subvoxel_of(const Scene& s, float x, float y, float z, int gs[3]) {
  const float q[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    float diff = q[a] - s.o32[a];
    float t = diff / s.hs32;
    float f = std::floor(t);
    int hi = s.dims[a] * s.p.dv - 1;
    int g = (f < 0.0f) ? 0 : (f > (float)hi ? hi : (int)f);
    gs[a] = g;
  }
}

struct Key {
  int64_t cell;
  int sub;
  int kind;
  uint32_t id;
  int64_t src;
};

// ------------------------------------------------------------------ Section 2.1: voxelisation
Scene* voxelize(const float* xyz, const float* nrm, const uint32_t* label, const uint8_t* material,
                int64_t n, const double* edges, const uint32_t* edge_label, int64_t n_edges,
                const double* region, const oracle_params* prm) {
  Scene* s = new Scene();
  s->p = *prm;
  s->h = prm->voxel_size;
  s->hs = prm->voxel_size / prm->dv;
  s->r_vox = s->h * std::sqrt(3.0) / 2.0;   // voxel bounding sphere (Section 2.2.4)
  s->r_sub = s->hs * std::sqrt(3.0) / 2.0;  // sphere encompassing an IE's subvoxel
  for (int64_t e = 0; e < n_edges; ++e) {
    const double* r = edges + 12 * e;
    Edge E;
    E.p0 = mk(r[0], r[1], r[2]);
    E.p1 = mk(r[3], r[4], r[5]);
    E.n0 = mk(r[6], r[7], r[8]);
    E.n1 = mk(r[9], r[10], r[11]);
    E.label = edge_label[e];
    s->edges.push_back(E);
  }
  // Grid: one voxel of padding below the bounds of the points, the edges and the
  // optional region box (region[0..2] min, region[3..5] max) that TX/RX must lie in.
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  if (region)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], region[a]);
      hi[a] = std::max(hi[a], region[3 + a]);
    }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], (double)xyz[3 * i + a]);
      hi[a] = std::max(hi[a], (double)xyz[3 * i + a]);
    }
  for (const Edge& E : s->edges)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], std::min(comp(E.p0, a), comp(E.p1, a)));
      hi[a] = std::max(hi[a], std::max(comp(E.p0, a), comp(E.p1, a)));
    }
  double org[3];
  for (int a = 0; a < 3; ++a) {
    org[a] = (std::floor(lo[a] / s->h) - 1.0) * s->h;
    s->dims[a] = (int)std::ceil((hi[a] - org[a]) / s->h) + 1;
    s->o32[a] = (float)org[a];
  }
  s->origin = mk(org[0], org[1], org[2]);
  s->hs32 = (float)s->hs;
  s->n_cells = (int64_t)s->dims[0] * s->dims[1] * s->dims[2];
  const int dv = prm->dv;

  auto key_of = [&](const int gs[3], int kind, uint32_t id, int64_t src) {
    Key k;
    k.cell = cell_of(*s, gs[0] / dv, gs[1] / dv, gs[2] / dv);
    k.sub = ((gs[2] % dv) * dv + (gs[1] % dv)) * dv + (gs[0] % dv);
    k.kind = kind;
    k.id = id;
    k.src = src;
    return k;
  };

  // Points: one entry per point, keyed by (voxel, subvoxel, label).
  std::vector<Key> keys;
  keys.reserve(n);
  for (int64_t i = 0; i < n; ++i) {
    int gs[3];
    subvoxel_of(*s, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], gs);
    keys.push_back(key_of(gs, IE_POINT, label[i], i));
  }
  // Edge segments inside subvoxels.  Reading: the edge is cut into fine pieces of
  // length <= h_s/4; a piece belongs to the subvoxel of its midpoint (binning rule
  // above) and consecutive pieces in one subvoxel form one edge IE whose reception
  // point is the midpoint of the joined segment.
  struct Piece { int edge; int64_t i0, i1, nf; int gs[3]; };
  std::vector<Piece> pieces;
  for (int64_t e = 0; e < n_edges; ++e) {
    const Edge& E = s->edges[e];
    double dx = E.p1.x - E.p0.x, dy = E.p1.y - E.p0.y, dz = E.p1.z - E.p0.z;
    double len = std::sqrt(dx * dx + dy * dy + dz * dz);
    int64_t nf = (int64_t)std::ceil(len / (s->hs / 4.0));
    if (nf < 1) nf = 1;
    int prev[3] = {-1, -1, -1};
    for (int64_t i = 0; i < nf; ++i) {
      double f = ((double)i + 0.5) / (double)nf;
      double m[3] = {E.p0.x + f * dx, E.p0.y + f * dy, E.p0.z + f * dz};
      int gs[3];
      subvoxel_of(*s, (float)m[0], (float)m[1], (float)m[2], gs);
      if (i == 0 || gs[0] != prev[0] || gs[1] != prev[1] || gs[2] != prev[2]) {
        Piece P;
        P.edge = (int)e; P.i0 = i; P.i1 = i; P.nf = nf;
        std::memcpy(P.gs, gs, sizeof gs);
        pieces.push_back(P);
      } else {
        pieces.back().i1 = i;
      }
      std::memcpy(prev, gs, sizeof gs);
    }
  }
  for (size_t k = 0; k < pieces.size(); ++k)
    keys.push_back(key_of(pieces[k].gs, IE_EDGE, (uint32_t)pieces[k].edge, (int64_t)k));

  std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    return std::tie(a.cell, a.sub, a.kind, a.id) < std::tie(b.cell, b.sub, b.kind, b.id);
  });

  // Group runs of equal keys into IEs.
  size_t i = 0;
  while (i < keys.size()) {
    size_t j = i;
    while (j < keys.size() && keys[j].cell == keys[i].cell && keys[j].sub == keys[i].sub &&
           keys[j].kind == keys[i].kind && keys[j].id == keys[i].id)
      ++j;
    IE ie;
    ie.kind = keys[i].kind;
    ie.cell = keys[i].cell;
    if (ie.kind == IE_POINT) {
      int64_t p0 = keys[i].src;
      subvoxel_of(*s, xyz[3 * p0], xyz[3 * p0 + 1], xyz[3 * p0 + 2], ie.gs);
      ie.label = keys[i].id;
      ie.material = 255;
      ie.p_begin = (int64_t)s->pts.size();
      ie.p_count = (int64_t)(j - i);
      V3 sum, nsum;
      V3 bmin = mk(1e300, 1e300, 1e300), bmax = mk(-1e300, -1e300, -1e300);
      for (size_t q = i; q < j; ++q) {
        int64_t src = keys[q].src;
        V3 P = mk(xyz[3 * src], xyz[3 * src + 1], xyz[3 * src + 2]);
        V3 N = mk(nrm[3 * src], nrm[3 * src + 1], nrm[3 * src + 2]);
        s->pts.push_back(P);
        s->nrm.push_back(N);
        sum = sum + P;
        nsum = nsum + N;
        bmin = mk(std::min(bmin.x, P.x), std::min(bmin.y, P.y), std::min(bmin.z, P.z));
        bmax = mk(std::max(bmax.x, P.x), std::max(bmax.y, P.y), std::max(bmax.z, P.z));
        ie.material = std::min<uint8_t>(ie.material, material ? material[src] : 0);
      }
      ie.rp = (1.0 / (double)(j - i)) * sum;  // reception point: centroid
      ie.normal = unit(nsum);                  // normalised mean normal
      ie.bbc = 0.5 * (bmin + bmax);
    } else {
      const Piece& P = pieces[keys[i].src];
      const Edge& E = s->edges[P.edge];
      std::memcpy(ie.gs, P.gs, sizeof P.gs);
      ie.label = E.label;
      ie.material = 255;
      ie.edge = P.edge;
      ie.t0 = (double)P.i0 / (double)P.nf;
      ie.t1 = (double)(P.i1 + 1) / (double)P.nf;
      double tm = 0.5 * (ie.t0 + ie.t1);
      ie.rp = E.p0 + tm * (E.p1 - E.p0);
      ie.normal = unit(E.n0 + E.n1);
      ie.bbc = ie.rp;
    }
    ie.sc = mk(s->origin.x + (ie.gs[0] + 0.5) * s->hs, s->origin.y + (ie.gs[1] + 0.5) * s->hs,
               s->origin.z + (ie.gs[2] + 0.5) * s->hs);
    s->ies.push_back(ie);
    i = j;
  }

  // Each low-resolution voxel knows its IEs (Section 2.1).
  s->cell_begin.assign(s->n_cells, 0);
  s->cell_count.assign(s->n_cells, 0);
  for (size_t k = 0; k < s->ies.size(); ++k) {
    int64_t c = s->ies[k].cell;
    if (s->cell_count[c] == 0) s->cell_begin[c] = (int64_t)k;
    s->cell_count[c] += 1;
  }

  // March distance (Section 2.2.4): the longest per-axis distance (L-infinity) to
  // the closest voxel that holds IEs; 0 for such voxels.  Multi-source
  // breadth-first search over the 26-neighbourhood gives exactly that distance.
  // Capped at 255 (and 255 when the grid holds no IE).
  s->march.assign(s->n_cells, 255);
  std::deque<int64_t> q;
  for (int64_t c = 0; c < s->n_cells; ++c)
    if (s->cell_count[c] > 0) { s->march[c] = 0; q.push_back(c); }
  while (!q.empty()) {
    int64_t c = q.front();
    q.pop_front();
    int vx = (int)(c % s->dims[0]), vy = (int)((c / s->dims[0]) % s->dims[1]),
        vz = (int)(c / ((int64_t)s->dims[0] * s->dims[1]));
    if (s->march[c] >= 255) continue;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!in_grid(*s, vx + dx, vy + dy, vz + dz)) continue;
          int64_t u = cell_of(*s, vx + dx, vy + dy, vz + dz);
          if (s->march[u] > s->march[c] + 1) { s->march[u] = s->march[c] + 1; q.push_back(u); }
        }
  }
  return s;
}

// ------------------------------------------------------- Section 2.2.1: point-set intersections
// Eq. 1: f(x) = (x - p(x)) . n(x), p and n the weighted averages of the IE's point
// positions and normals.  Reading: Gaussian weights exp(-|x-p_i|^2 / sigma^2) over
// the points of the IE being intersected.  Returns false when every weight is 0.
bool sdf_eval(const Scene& s, const IE& ie, V3 x, double* f, V3* n_out) {
  const double inv_s2 = 1.0 / (s.p.sdf_sigma * s.p.sdf_sigma);
  double sw = 0.0;
  V3 sp, sn;
  for (int64_t k = 0; k < ie.p_count; ++k) {
    const V3& P = s.pts[ie.p_begin + k];
    V3 d = x - P;
    double w = std::exp(-dot(d, d) * inv_s2);
    sw += w;
    sp = sp + w * P;
    sn = sn + w * s.nrm[ie.p_begin + k];
  }
  if (!(sw > 0.0)) return false;
  V3 p = (1.0 / sw) * sp;
  double nn = norm(sn);
  if (!(nn > 0.0)) return false;
  V3 n = (1.0 / nn) * sn;
  *f = dot(x - p, n);
  if (n_out) *n_out = n;
  return true;
}

// Ray / point-set intersection (Section 2.2.1).  The bounding-box centre is
// projected onto the ray; a segment of the subvoxel's diameter is centred there.
// From the end nearest the ray origin, advance by |f(s_i)| until the sign of f
// changes or |f| is near zero (hit), or the segment end is passed (miss).
// Readings: at most sdf_max_steps steps (then miss); the hit is placed by a secant
// step on a sign change and by one Newton step along the ray otherwise.
bool sdf_hit(const Scene& s, const IE& ie, V3 P, V3 d, double* t_hit) {
  const double L = s.hs * std::sqrt(3.0);
  double tc = dot(ie.bbc - P, d);
  double t = tc - 0.5 * L, t_end = tc + 0.5 * L;
  double f;
  V3 n;
  if (!sdf_eval(s, ie, P + t * d, &f, &n)) return false;
  for (int it = 0; it < s.p.sdf_max_steps; ++it) {
    if (std::fabs(f) < s.p.sdf_eps) {
      double dn = dot(n, d);
      double th = std::fabs(dn) > 1e-3 ? t - f / dn : t;
      // reading: the intersection lies on the marched segment; a Newton placement
      // past either end (grazing rays) is not an intersection of this point set
      if (th < tc - 0.5 * L || th > t_end) return false;
      *t_hit = th;
      return true;
    }
    double t_next = t + std::fabs(f);
    if (t_next > t_end) return false;
    double f_next;
    V3 n_next;
    if (!sdf_eval(s, ie, P + t_next * d, &f_next, &n_next)) return false;
    if ((f_next < 0.0) != (f < 0.0)) {
      *t_hit = t - f * (t_next - t) / (f_next - f);
      return true;
    }
    t = t_next;
    f = f_next;
    n = n_next;
  }
  return false;
}

// --------------------------------------------------------------------------- traversal
// Voxel traversal of the ray P + t d, t in [0, t_end] (Amanatides-Woo); ties of the
// next boundary pick the lowest axis.  visit() returns false to stop.
template <class F>
void dda(const Scene& s, V3 P, V3 d, double t_end, F&& visit) {
  int v[3], step[3];
  double tmax[3], tdelta[3];
  for (int a = 0; a < 3; ++a) {
    double o = comp(s.origin, a), pa = comp(P, a), da = comp(d, a);
    v[a] = (int)std::floor((pa - o) / s.h);
    if (v[a] < 0 || v[a] >= s.dims[a]) return;
    if (da > 0) {
      step[a] = 1; tmax[a] = (o + (v[a] + 1) * s.h - pa) / da; tdelta[a] = s.h / da;
    } else if (da < 0) {
      step[a] = -1; tmax[a] = (o + v[a] * s.h - pa) / da; tdelta[a] = -s.h / da;
    } else {
      step[a] = 0; tmax[a] = std::numeric_limits<double>::infinity();
      tdelta[a] = std::numeric_limits<double>::infinity();
    }
  }
  for (;;) {
    if (!visit(v)) return;
    int a = 0;
    if (tmax[1] < tmax[a]) a = 1;
    if (tmax[2] < tmax[a]) a = 2;
    if (tmax[a] > t_end) return;
    v[a] += step[a];
    if (v[a] < 0 || v[a] >= s.dims[a]) return;
    tmax[a] += tdelta[a];
  }
}

// Endpoint self-hit rule (reading): a hit within vis_ignore of a path node is not an
// occlusion when it lies on that node's own surface (point IE: same label) or, at an
// edge, on any surface (the faces meeting there).  TX and RX ignore nothing.
enum { IGN_NONE = 0, IGN_LABEL = 1, IGN_ANY = 2 };
struct Endpoint {
  int mode;
  uint32_t label;
};

bool ignored(const Endpoint& e, uint32_t lbl, double dist, double r) {
  if (dist >= r) return false;
  if (e.mode == IGN_ANY) return true;
  if (e.mode == IGN_LABEL) return lbl == e.label;
  return false;
}

bool segment_sphere(V3 A, V3 d, double T, V3 C, double r) {
  double tc = std::min(std::max(dot(C - A, d), 0.0), T);
  V3 q = A + tc * d - C;
  return dot(q, q) <= r * r;
}

// Occlusion test of one point IE against the segment A -> B.
bool ie_blocks(const Scene& s, const IE& ie, V3 A, V3 d, double T, Endpoint ea, Endpoint eb) {
  if (ie.kind != IE_POINT) return false;  // edges and RXs never occlude
  if (!segment_sphere(A, d, T, ie.sc, s.r_sub)) return false;
  double t;
  if (!sdf_hit(s, ie, A, d, &t)) return false;
  if (!(t > 0.0 && t < T)) return false;
  double r = s.p.vis_ignore;
  if (ignored(ea, ie.label, t, r) || ignored(eb, ie.label, T - t, r)) return false;
  return true;
}

// Visibility (Sections 2.2.4 and 2.3): trace a ray from A to B through the voxel grid
// and test the point IEs of every voxel it passes.
bool visible(const Scene& s, V3 A, V3 B, Endpoint ea, Endpoint eb, int64_t* n_tests = nullptr) {
  V3 dv = B - A;
  double T = norm(dv);
  if (T < 1e-12) return true;
  V3 d = (1.0 / T) * dv;
  bool vis = true;
  dda(s, A, d, T, [&](const int v[3]) {
    int64_t c = cell_of(s, v[0], v[1], v[2]);
    for (int32_t k = 0; k < s.cell_count[c]; ++k) {
      if (n_tests) ++*n_tests;
      if (ie_blocks(s, s.ies[s.cell_begin[c] + k], A, d, T, ea, eb)) { vis = false; return false; }
    }
    return true;
  });
  return vis;
}

// The same test without the traversal: the voxels the segment passes are found by
// a slab test against every voxel of the grid (brute force, for tiny scenes).
bool visible_bruteforce(const Scene& s, V3 A, V3 B, Endpoint ea, Endpoint eb) {
  V3 dv = B - A;
  double T = norm(dv);
  if (T < 1e-12) return true;
  V3 d = (1.0 / T) * dv;
  for (int vz = 0; vz < s.dims[2]; ++vz)
    for (int vy = 0; vy < s.dims[1]; ++vy)
      for (int vx = 0; vx < s.dims[0]; ++vx) {
        int64_t c = cell_of(s, vx, vy, vz);
        if (s.cell_count[c] == 0) continue;
        double t0 = 0.0, t1 = T;
        int vv[3] = {vx, vy, vz};
        bool hit = true;
        for (int a = 0; a < 3 && hit; ++a) {
          double lo = comp(s.origin, a) + vv[a] * s.h, hi = lo + s.h;
          double pa = comp(A, a), da = comp(d, a);
          if (da == 0.0) {
            if (pa < lo || pa >= hi) hit = false;
          } else {
            double ta = (lo - pa) / da, tb = (hi - pa) / da;
            if (ta > tb) std::swap(ta, tb);
            t0 = std::max(t0, ta);
            t1 = std::min(t1, tb);
            if (t0 > t1) hit = false;
          }
        }
        if (!hit) continue;
        for (int32_t k = 0; k < s.cell_count[c]; ++k)
          if (ie_blocks(s, s.ies[s.cell_begin[c] + k], A, d, T, ea, eb)) return false;
      }
  return true;
}

// ------------------------------------------------------------------ Section 2.2.4: cones
// Cone-sphere test: the sphere (C, r) meets the one-sided cone (apex, unit axis,
// half-angle alpha) iff the angle between the axis and C - apex is at most
// alpha + asin(r/|C - apex|), written without trigonometry.
bool cone_sphere(V3 apex, V3 axis, double sin_a, double cos_a, V3 C, double r) {
  V3 v = C - apex;
  double d2 = dot(v, v);
  if (d2 <= r * r) return true;
  double t = dot(v, axis);
  return t + r * sin_a >= cos_a * std::sqrt(d2 - r * r);
}

enum { CONE_PRIMARY = 0, CONE_REFLECT = 1, CONE_DIFFRACT = 2 };

struct Cone {
  V3 apex, axis;
  double sin_a = 0, cos_a = 1;
  int kind = CONE_PRIMARY;
  V3 pn;               // reflection: separation plane normal (oriented surface normal)
  V3 tlo, thi, rmid;   // diffraction: the two separation planes and the mid direction
  Endpoint origin;     // self-hit rule of the apex
};

// Separation planes (Section 2.2.4).  Reading for reflections: the plane through the
// apex tangent to the reflecting surface; an IE must lie more than sep_eps in front
// of it.  Diffraction: the planes through the edge half-way to the neighbouring fan
// rays; the reception point must lie between them (and on this ray's side).
bool passes_planes(const Scene& s, const Cone& c, V3 q) {
  V3 r = q - c.apex;
  if (c.kind == CONE_REFLECT) return dot(r, c.pn) > s.p.sep_eps;
  if (c.kind == CONE_DIFFRACT) return dot(r, c.tlo) >= 0.0 && dot(r, c.thi) < 0.0 && dot(r, c.rmid) > 0.0;
  return true;
}

struct TraceCtx {
  const Scene* s;
  std::vector<V3> rx;
  std::vector<V3> rx_sc;
  std::map<int64_t, std::vector<int>> rx_in_cell;
  std::vector<int32_t> march;   // scene march distance with the RX voxels included
  int64_t n_cones = 0, n_vis = 0, n_evals = 0;
};

struct MarchResult {
  std::vector<int64_t> ies;                 // accepted point / edge IEs
  std::vector<std::pair<int, double>> rx;   // accepted RXs and their miss distance
};

// Voxel cone tracing (Section 2.2.4).  The cone's axis is traversed voxel by voxel.
// Where the march distance is at most 1 (the voxel or a neighbour holds IEs), the
// neighbouring voxels are evaluated: voxel bounding sphere vs cone, then each IE's
// subvoxel sphere vs cone, the separation planes, and a visibility ray from the
// apex to the reception point.  Readings: a neighbourhood already evaluated for
// this cone is not evaluated again; the cone stops after the first evaluation that
// accepts a point IE (RX and edge IEs never stop it); edge IEs are only tested
// when the node may still diffract.
MarchResult march_cone(TraceCtx& ctx, const Cone& cone, bool test_edges) {
  const Scene& s = *ctx.s;
  MarchResult res;
  ctx.n_cones++;
  bool have_last = false;
  int last[3] = {0, 0, 0};
  dda(s, cone.apex, cone.axis, std::numeric_limits<double>::infinity(), [&](const int v[3]) {
    if (ctx.march[cell_of(s, v[0], v[1], v[2])] > 1) return true;
    ctx.n_evals++;
    std::vector<int64_t> cand;
    std::vector<int> rcand;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int u[3] = {v[0] + dx, v[1] + dy, v[2] + dz};
          if (!in_grid(s, u[0], u[1], u[2])) continue;
          if (have_last && std::abs(u[0] - last[0]) <= 1 && std::abs(u[1] - last[1]) <= 1 &&
              std::abs(u[2] - last[2]) <= 1)
            continue;
          int64_t c = cell_of(s, u[0], u[1], u[2]);
          auto rit = ctx.rx_in_cell.find(c);
          bool has_rx = rit != ctx.rx_in_cell.end();
          if (s.cell_count[c] == 0 && !has_rx) continue;
          if (!cone_sphere(cone.apex, cone.axis, cone.sin_a, cone.cos_a, voxel_center(s, u[0], u[1], u[2]), s.r_vox))
            continue;
          for (int32_t k = 0; k < s.cell_count[c]; ++k) {
            int64_t id = s.cell_begin[c] + k;
            const IE& ie = s.ies[id];
            if (ie.kind == IE_EDGE && !test_edges) continue;
            if (!cone_sphere(cone.apex, cone.axis, cone.sin_a, cone.cos_a, ie.sc, s.r_sub)) continue;
            if (!passes_planes(s, cone, ie.rp)) continue;
            cand.push_back(id);
          }
          if (has_rx)
            for (int j : rit->second) {
              if (!cone_sphere(cone.apex, cone.axis, cone.sin_a, cone.cos_a, ctx.rx_sc[j], s.r_sub)) continue;
              if (!passes_planes(s, cone, ctx.rx[j])) continue;
              rcand.push_back(j);
            }
        }
    have_last = true;
    std::memcpy(last, v, sizeof last);
    bool stop = false;
    for (int64_t id : cand) {
      const IE& ie = s.ies[id];
      Endpoint eb{ie.kind == IE_EDGE ? IGN_ANY : IGN_LABEL, ie.label};
      ctx.n_vis++;
      if (visible(s, cone.apex, ie.rp, cone.origin, eb)) {
        res.ies.push_back(id);
        if (ie.kind == IE_POINT) stop = true;
      }
    }
    for (int j : rcand) {
      ctx.n_vis++;
      if (visible(s, cone.apex, ctx.rx[j], cone.origin, Endpoint{IGN_NONE, NONE_LABEL})) {
        V3 r = ctx.rx[j] - cone.apex;
        V3 perp = r - dot(r, cone.axis) * cone.axis;
        res.rx.push_back({j, norm(perp)});
      }
    }
    return !stop;
  });
  return res;
}

// Uniform launch directions: a Fibonacci lattice of N points on the unit sphere
// (equal-area spiral: z_i = 1 - (2i+1)/N, azimuth i times the golden angle).
void fibonacci_dir(int64_t i, int64_t N, double out[3]) {
  const double golden = PI * (3.0 - std::sqrt(5.0));
  double z = 1.0 - (2.0 * (double)i + 1.0) / (double)N;
  double r = std::sqrt(std::max(0.0, 1.0 - z * z));
  double phi = std::fmod((double)i * golden, 2.0 * PI);
  out[0] = r * std::cos(phi);
  out[1] = r * std::sin(phi);
  out[2] = z;
}

struct Node {
  int tx;
  int64_t parent;     // index into the node store, -1 for the TX
  int64_t ie;
  int type;
  int depth, nr, nd;
  V3 apex, in_dir;
};

struct Coarse {
  int tx, rx, n;
  int64_t ie[MAXI];
  int type[MAXI];
  uint32_t label[MAXI];
  double miss;
};

struct CoarseSet {
  std::vector<Coarse> paths;     // after the kappa selection
  int64_t n_before_kappa = 0;
  int64_t n_cones = 0, n_vis = 0, n_evals = 0;
  std::vector<int64_t> nodes_per_level;
  std::vector<V3> tx, rx;
};

// Cones cast from a node (Sections 2.2.3-2.2.4).  Reflection: one cone whose axis is
// the incoming direction mirrored about the IE normal (normal turned toward the
// incoming side).  Diffraction: a fan on Keller's cone about the edge -- rays at
// the incoming angle beta to the edge, azimuths phi_j = j * 2pi/M with
// M = ceil(pi/alpha) (spacing 2 alpha), kept where they point out of the wedge
// (exterior edges only, Section 3.2).
std::vector<Cone> cones_of(const Scene& s, const Node& nd, double alpha) {
  std::vector<Cone> out;
  const IE& ie = s.ies[nd.ie];
  V3 e = nd.in_dir;
  if (nd.type == T_REFL) {
    Cone c;
    c.kind = CONE_REFLECT;
    c.apex = ie.rp;
    V3 n = ie.normal;
    if (dot(n, e) > 0) n = -1.0 * n;
    c.axis = unit(e - 2.0 * dot(e, n) * n);
    c.pn = n;
    c.sin_a = std::sin(alpha);
    c.cos_a = std::cos(alpha);
    c.origin = Endpoint{IGN_LABEL, ie.label};
    out.push_back(c);
    return out;
  }
  const Edge& E = s.edges[ie.edge];
  V3 w = unit(E.p1 - E.p0);
  double cb = dot(e, w);
  double sb2 = 1.0 - cb * cb;
  if (sb2 < 1e-12) return out;
  double sb = std::sqrt(sb2);
  V3 a, b;
  onb(w, &a, &b);
  int M = (int)std::ceil(PI / alpha);
  double dphi = 2.0 * PI / M;
  for (int j = 0; j < M; ++j) {
    double phi = j * dphi;
    V3 r = std::cos(phi) * a + std::sin(phi) * b;
    V3 d = cb * w + sb * r;
    if (!(dot(d, E.n0) > 0.0 || dot(d, E.n1) > 0.0)) continue;
    Cone c;
    c.kind = CONE_DIFFRACT;
    c.apex = ie.rp;
    c.axis = unit(d);
    c.sin_a = std::sin(alpha);
    c.cos_a = std::cos(alpha);
    double plo = phi - 0.5 * dphi, phi_hi = phi + 0.5 * dphi;
    c.tlo = -std::sin(plo) * a + std::cos(plo) * b;
    c.thi = -std::sin(phi_hi) * a + std::cos(phi_hi) * b;
    c.rmid = r;
    c.origin = Endpoint{IGN_ANY, ie.label};
    out.push_back(c);
  }
  return out;
}

// ---------------------------------------------------------- Section 2.2: coarse path tracing
CoarseSet* trace(const Scene& s, const double* txp, int ntx, const double* rxp, int nrx) {
  const oracle_params& p = s.p;
  CoarseSet* out = new CoarseSet();
  TraceCtx ctx;
  ctx.s = &s;
  for (int j = 0; j < nrx; ++j) {
    V3 r = mk(rxp[3 * j], rxp[3 * j + 1], rxp[3 * j + 2]);
    int gs[3];
    subvoxel_of(s, (float)r.x, (float)r.y, (float)r.z, gs);
    int dv = p.dv;
    ctx.rx.push_back(r);
    // Reading: an RX entity's reception sphere (radius of the subvoxel sphere) is
    // centred on the RX itself, so reception does not depend on where the RX
    // falls inside its subvoxel.
    ctx.rx_sc.push_back(r);
    ctx.rx_in_cell[cell_of(s, gs[0] / dv, gs[1] / dv, gs[2] / dv)].push_back(j);
    out->rx.push_back(r);
  }
  for (int t = 0; t < ntx; ++t) out->tx.push_back(mk(txp[3 * t], txp[3 * t + 1], txp[3 * t + 2]));
  // RX entities are IEs too: their voxels count as holding IEs for the march distance.
  ctx.march = s.march;
  for (int64_t c = 0; c < s.n_cells; ++c) {
    int vx = (int)(c % s.dims[0]), vy = (int)((c / s.dims[0]) % s.dims[1]),
        vz = (int)(c / ((int64_t)s.dims[0] * s.dims[1]));
    for (auto& kv : ctx.rx_in_cell) {
      int64_t rc = kv.first;
      int rx_ = (int)(rc % s.dims[0]), ry = (int)((rc / s.dims[0]) % s.dims[1]),
          rz = (int)(rc / ((int64_t)s.dims[0] * s.dims[1]));
      int dist = std::max(std::abs(vx - rx_), std::max(std::abs(vy - ry), std::abs(vz - rz)));
      ctx.march[c] = std::min(ctx.march[c], dist);
    }
  }
  const int max_int = p.max_int;
  const double alpha = p.cone_half_angle;
  const double alpha0 = std::max(alpha, p.launch_spacing / std::sqrt(2.0));
  const int64_t nl = p.n_launch;

  std::vector<Node> store;
  std::vector<Coarse> raw;
  auto chain_of = [&](int64_t node, Coarse& c) {
    int n = store[node].depth;
    c.n = n;
    int64_t k = node;
    for (int q = n - 1; q >= 0; --q) {
      const Node& nd = store[k];
      c.ie[q] = nd.ie;
      c.type[q] = nd.type;
      c.label[q] = s.ies[nd.ie].label;
      k = nd.parent;
    }
  };

  std::vector<int64_t> frontier;
  // Transmission phase (Section 2.2.2).  Uniform launch reading (launch_mode 0):
  // cones on a Fibonacci lattice from each TX; the IEs they accept are the initial
  // interactions (a set per TX) and the RXs they accept are LOS connections.  The
  // paper's own launch (launch_mode 1): a ray from the TX toward every IE (edge IEs
  // only when a diffraction is allowed) and every RX; the visible ones are the
  // initial interactions and the LOS connections (the ray points at the RX: miss 0).
  for (int t = 0; t < ntx; ++t) {
    V3 T = out->tx[t];
    std::set<int64_t> first;
    std::map<int, double> los;
    if (p.launch_mode == 1) {
      const bool test_edges = max_int >= 1 && p.max_diff >= 1;
      for (int64_t id = 0; id < (int64_t)s.ies.size(); ++id) {
        const IE& ie = s.ies[id];
        if (ie.kind == IE_EDGE && !test_edges) continue;
        ctx.n_vis++;
        if (visible(s, T, ie.rp, Endpoint{IGN_NONE, NONE_LABEL},
                    Endpoint{ie.kind == IE_EDGE ? IGN_ANY : IGN_LABEL, ie.label}))
          first.insert(id);
      }
      for (int j = 0; j < nrx; ++j) {
        ctx.n_vis++;
        if (visible(s, T, out->rx[j], Endpoint{IGN_NONE, NONE_LABEL}, Endpoint{IGN_NONE, NONE_LABEL})) los[j] = 0.0;
      }
    }
    for (int64_t i = 0; i < (p.launch_mode == 1 ? 0 : nl); ++i) {
      double d[3];
      fibonacci_dir(i, nl, d);
      Cone c;
      c.kind = CONE_PRIMARY;
      c.apex = T;
      c.axis = mk(d[0], d[1], d[2]);
      c.sin_a = std::sin(alpha0);
      c.cos_a = std::cos(alpha0);
      c.origin = Endpoint{IGN_NONE, NONE_LABEL};
      bool test_edges = max_int >= 1 && p.max_diff >= 1;
      MarchResult r = march_cone(ctx, c, test_edges);
      for (int64_t id : r.ies) first.insert(id);
      for (auto& h : r.rx) {
        auto it = los.find(h.first);
        if (it == los.end() || h.second < it->second) los[h.first] = h.second;
      }
    }
    for (auto& kv : los) {
      Coarse c;
      std::memset(&c, 0, sizeof c);
      c.tx = t;
      c.rx = kv.first;
      c.n = 0;
      c.miss = kv.second;
      raw.push_back(c);
    }
    if (max_int < 1) continue;
    for (int64_t id : first) {
      const IE& ie = s.ies[id];
      Node nd;
      nd.tx = t; nd.parent = -1; nd.ie = id; nd.depth = 1;
      nd.type = ie.kind == IE_EDGE ? T_DIFF : T_REFL;
      nd.nr = nd.type == T_REFL; nd.nd = nd.type == T_DIFF;
      if (nd.nr > p.max_refl || nd.nd > p.max_diff) continue;
      nd.apex = ie.rp;
      nd.in_dir = unit(ie.rp - T);
      store.push_back(nd);
      frontier.push_back((int64_t)store.size() - 1);
    }
  }
  out->nodes_per_level.push_back((int64_t)frontier.size());
  // Propagation phase (Section 2.2.3): rays leave each interaction point, reflected
  // or diffracted, until no IE is hit or the interaction limit is reached.
  while (!frontier.empty()) {
    std::vector<int64_t> next;
    for (int64_t ni : frontier) {
      Node nd = store[ni];
      bool can_child = nd.depth < max_int;
      bool test_edges = can_child && nd.nd < p.max_diff;
      std::vector<Cone> cones = cones_of(s, nd, alpha);
      for (const Cone& c : cones) {
        MarchResult r = march_cone(ctx, c, test_edges);
        for (auto& h : r.rx) {
          Coarse cp;
          std::memset(&cp, 0, sizeof cp);
          cp.tx = nd.tx;
          cp.rx = h.first;
          cp.miss = h.second;
          chain_of(ni, cp);
          raw.push_back(cp);
        }
        if (!can_child) continue;
        for (int64_t id : r.ies) {
          const IE& ie = s.ies[id];
          Node ch;
          ch.tx = nd.tx; ch.parent = ni; ch.ie = id; ch.depth = nd.depth + 1;
          ch.type = ie.kind == IE_EDGE ? T_DIFF : T_REFL;
          ch.nr = nd.nr + (ch.type == T_REFL);
          ch.nd = nd.nd + (ch.type == T_DIFF);
          if (ch.nr > p.max_refl || ch.nd > p.max_diff) continue;
          ch.apex = ie.rp;
          ch.in_dir = unit(ie.rp - nd.apex);
          store.push_back(ch);
          next.push_back((int64_t)store.size() - 1);
        }
      }
    }
    if (!next.empty()) out->nodes_per_level.push_back((int64_t)next.size());
    frontier.swap(next);
  }
  out->n_before_kappa = (int64_t)raw.size();
  // Duplicate limit kappa (Section 2.2.3): at most kappa coarse paths with the same
  // labels in the same order, per TX/RX pair.  Reading: keep those whose last cone
  // axis passes nearest the RX, ties broken by the IE sequence.
  auto group_less = [](const Coarse& a, const Coarse& b) {
    if (a.tx != b.tx) return a.tx < b.tx;
    if (a.rx != b.rx) return a.rx < b.rx;
    if (a.n != b.n) return a.n < b.n;
    for (int q = 0; q < a.n; ++q) {
      if (a.type[q] != b.type[q]) return a.type[q] < b.type[q];
      if (a.label[q] != b.label[q]) return a.label[q] < b.label[q];
    }
    return false;
  };
  std::sort(raw.begin(), raw.end(), [&](const Coarse& a, const Coarse& b) {
    if (group_less(a, b)) return true;
    if (group_less(b, a)) return false;
    if (a.miss != b.miss) return a.miss < b.miss;
    for (int q = 0; q < a.n; ++q)
      if (a.ie[q] != b.ie[q]) return a.ie[q] < b.ie[q];
    return false;
  });
  size_t g = 0;
  while (g < raw.size()) {
    size_t h = g;
    while (h < raw.size() && !group_less(raw[g], raw[h]) && !group_less(raw[h], raw[g])) ++h;
    for (size_t q = g; q < h && (int)(q - g) < p.kappa; ++q) out->paths.push_back(raw[q]);
    g = h;
  }
  out->n_cones = ctx.n_cones;
  out->n_vis = ctx.n_vis;
  out->n_evals = ctx.n_evals;
  return out;
}

// ------------------------------------------------------------- Section 2.3: refinement
struct Exact {
  int tx, rx, n;
  int type[MAXI];
  uint32_t label[MAXI];
  uint8_t material[MAXI];
  int64_t ie[MAXI];
  V3 pts[MAXI];
  double length, delay, grad;
  int iters, status;
  int64_t coarse;
};

enum { ST_VALID = 0, ST_MISS = 1, ST_NOT_CONVERGED = 2, ST_OCCLUDED = 3, ST_OFF_EDGE = 4 };

// Eq. 1 over the nearby points of one surface.  Reading: "nearby" = the points of
// label `label` whose subvoxel lies in the 3x3x3 block of subvoxels around the
// subvoxel of x, so the implicit surface of a label is continuous across subvoxel
// boundaries (the re-projection below needs that to converge on noisy clouds).
bool sdf_label(const Scene& s, uint32_t label, V3 x, double* f, V3* n_out) {
  const int dv = s.p.dv;
  int g[3], v0[3], v1[3];
  for (int a = 0; a < 3; ++a) {
    g[a] = (int)std::floor((comp(x, a) - comp(s.origin, a)) / s.hs);
    v0[a] = (int)std::floor((double)(g[a] - 1) / dv);
    v1[a] = (int)std::floor((double)(g[a] + 1) / dv);
  }
  const double inv_s2 = 1.0 / (s.p.sdf_sigma * s.p.sdf_sigma);
  double sw = 0.0;
  V3 sp, sn;
  for (int vz = v0[2]; vz <= v1[2]; ++vz)
    for (int vy = v0[1]; vy <= v1[1]; ++vy)
      for (int vx = v0[0]; vx <= v1[0]; ++vx) {
        if (!in_grid(s, vx, vy, vz)) continue;
        int64_t c = cell_of(s, vx, vy, vz);
        for (int32_t k = 0; k < s.cell_count[c]; ++k) {
          const IE& ie = s.ies[s.cell_begin[c] + k];
          if (ie.kind != IE_POINT || ie.label != label) continue;
          if (std::abs(ie.gs[0] - g[0]) > 1 || std::abs(ie.gs[1] - g[1]) > 1 || std::abs(ie.gs[2] - g[2]) > 1)
            continue;
          for (int64_t q = 0; q < ie.p_count; ++q) {
            const V3& P = s.pts[ie.p_begin + q];
            V3 d = x - P;
            double w = std::exp(-dot(d, d) * inv_s2);
            sw += w;
            sp = sp + w * P;
            sn = sn + w * s.nrm[ie.p_begin + q];
          }
        }
      }
  if (!(sw > 0.0)) return false;
  double nn = norm(sn);
  if (!(nn > 0.0)) return false;
  V3 n = (1.0 / nn) * sn;
  *f = dot(x - (1.0 / sw) * sp, n);
  if (n_out) *n_out = n;
  return true;
}

// Re-projection (Section 2.3): a ray from the previous interaction point toward the
// updated reflection point R; its intersection with the surface of label l gives the
// new c_k, and the normal there (Eq. 1 normal) the new u_k, v_k.  The intersection is
// sought on a segment of one subvoxel diameter centred on R.  Reading: Eq. 1 is
// evaluated at R first; where R already lies on the surface (|f(R)| < eps) the hit is
// one Newton step along the ray from R, as at the end of a march, if that stays on
// the segment, and its normal is Eq. 1's at R (the two points coincide once the path
// is stationary).  Otherwise the segment is marched from its near end (Section
// 2.2.1) and the normal is taken at the hit.
bool reproject(const Scene& s, V3 P, V3 R, uint32_t label, V3* c_out, V3* n_out) {
  V3 dvec = R - P;
  double tR = norm(dvec);
  if (tR < 1e-12) return false;
  V3 d = (1.0 / tR) * dvec;
  const double L = s.hs * std::sqrt(3.0);
  double t = tR - 0.5 * L, t_end = tR + 0.5 * L, th = 0.0;
  double f;
  V3 n;
  bool hit = false;
  {
    double fR;
    V3 nR;
    if (sdf_label(s, label, R, &fR, &nR) && std::fabs(fR) < s.p.sdf_eps) {
      double dn = dot(nR, d);
      double tR_hit = std::fabs(dn) > 1e-3 ? tR - fR / dn : tR;
      if (tR_hit > 0.0 && std::fabs(tR_hit - tR) <= 0.5 * L) {
        *c_out = P + tR_hit * d;
        *n_out = nR;
        return true;
      }
    }
  }
  if (!sdf_label(s, label, P + t * d, &f, &n)) return false;
  for (int it = 0; it < s.p.sdf_max_steps && !hit; ++it) {
    if (std::fabs(f) < s.p.sdf_eps) {
      double dn = dot(n, d);
      th = std::fabs(dn) > 1e-3 ? t - f / dn : t;
      hit = true;
      break;
    }
    double t_next = t + std::fabs(f);
    if (t_next > t_end) return false;
    double f_next;
    V3 n_next;
    if (!sdf_label(s, label, P + t_next * d, &f_next, &n_next)) return false;
    if ((f_next < 0.0) != (f < 0.0)) {
      th = t - f * (t_next - t) / (f_next - f);
      hit = true;
      break;
    }
    t = t_next;
    f = f_next;
    n = n_next;
  }
  // the placed hit must stay on the marched segment
  if (!hit || !(th > 0.0) || std::fabs(th - tR) > 0.5 * L) return false;
  V3 c = P + th * d;
  if (!sdf_label(s, label, c, &f, &n)) return false;
  *c_out = c;
  *n_out = n;
  return true;
}

// Gradient of Eq. 2 with respect to the local variables: for reflection k,
// df_k/dr_k = (e_in + e_out).u_k and df_k/ds_k = (e_in + e_out).v_k; for diffraction k,
// df_k/dt_k = (e_in + e_out).w_k, with e_in = (I_k - I_{k-1})/|.|, e_out = (I_k - I_{k+1})/|.|.
void gradient(int n, const V3* I, const int* type, const V3* u, const V3* v, const V3* w, double g[][2]) {
  for (int k = 1; k <= n; ++k) {
    V3 e = unit(I[k] - I[k - 1]) + unit(I[k] - I[k + 1]);
    if (type[k - 1] == T_REFL) {
      g[k][0] = dot(e, u[k]);
      g[k][1] = dot(e, v[k]);
    } else {
      g[k][0] = dot(e, w[k]);
      g[k][1] = 0.0;
    }
  }
}

Exact refine_one(const Scene& s, const CoarseSet& cs, const Coarse& cp) {
  const oracle_params& p = s.p;
  Exact ex;
  std::memset(&ex, 0, sizeof ex);
  ex.tx = cp.tx; ex.rx = cp.rx; ex.n = cp.n;
  const int n = cp.n;
  V3 I[MAXI + 2], c[MAXI + 2], nrm[MAXI + 2], u[MAXI + 2], v[MAXI + 2], w[MAXI + 2];
  double tpar[MAXI + 2] = {0}, elen[MAXI + 2] = {0};
  I[0] = cs.tx[cp.tx];
  I[n + 1] = cs.rx[cp.rx];
  for (int k = 1; k <= n; ++k) {
    const IE& ie = s.ies[cp.ie[k - 1]];
    ex.type[k - 1] = cp.type[k - 1];
    ex.label[k - 1] = cp.label[k - 1];
    ex.material[k - 1] = ie.material;
    ex.ie[k - 1] = cp.ie[k - 1];
    c[k] = ie.rp;
    I[k] = ie.rp;
    if (cp.type[k - 1] == T_REFL) {
      nrm[k] = ie.normal;
      onb(nrm[k], &u[k], &v[k]);
    } else {
      const Edge& E = s.edges[ie.edge];
      w[k] = unit(E.p1 - E.p0);
      elen[k] = norm(E.p1 - E.p0);
    }
  }
  double g[MAXI + 2][2] = {{0}};
  bool converged = false;
  int it = 0;
  double gn = 0;
  for (; it < p.rho; ++it) {
    gradient(n, I, cp.type, u, v, w, g);
    double g2 = 0;
    for (int k = 1; k <= n; ++k) g2 += g[k][0] * g[k][0] + g[k][1] * g[k][1];
    gn = std::sqrt(g2);
    if (gn < p.grad_stop) { converged = true; break; }
    V3 In[MAXI + 2];
    In[0] = I[0];
    In[n + 1] = I[n + 1];
    // Gradient-descent step, reading: each interaction's gradient is scaled by the
    // inverse Hessian of its own local length f_k (2x2 in (r, s), 1x1 in t) times
    // gamma, with all interactions updated from the same iterate (Jacobi); where that
    // Hessian is near singular the step is gamma / (1/a + 1/b) times the gradient.
    // The stationary points, and so the exact paths, do not depend on this choice.
    for (int k = 1; k <= n; ++k) {
      double a = norm(I[k] - I[k - 1]), b = norm(I[k] - I[k + 1]);
      double eta = p.gamma / (1.0 / a + 1.0 / b);
      double hsc = (1.0 / a + 1.0 / b) * (1.0 / a + 1.0 / b);
      V3 ea = unit(I[k] - I[k - 1]), eb = unit(I[k] - I[k + 1]);
      if (cp.type[k - 1] == T_REFL) {
        double au = dot(ea, u[k]), av = dot(ea, v[k]), bu = dot(eb, u[k]), bv = dot(eb, v[k]);
        double h11 = (1.0 - au * au) / a + (1.0 - bu * bu) / b;
        double h22 = (1.0 - av * av) / a + (1.0 - bv * bv) / b;
        double h12 = -(au * av) / a - (bu * bv) / b;
        double det = h11 * h22 - h12 * h12;
        double r, sv;
        if (det > 1e-12 * hsc) {
          r = -p.gamma * (h22 * g[k][0] - h12 * g[k][1]) / det;
          sv = -p.gamma * (h11 * g[k][1] - h12 * g[k][0]) / det;
        } else {
          r = -eta * g[k][0];
          sv = -eta * g[k][1];
        }
        double len = std::sqrt(r * r + sv * sv);
        if (len > s.hs) { r *= s.hs / len; sv *= s.hs / len; }
        V3 R = c[k] + r * u[k] + sv * v[k];      // R_k = c_k + r_k u_k + s_k v_k
        V3 cn, nn;
        if (!reproject(s, I[k - 1], R, cp.label[k - 1], &cn, &nn)) {
          ex.status = ST_MISS; ex.iters = it; ex.grad = gn;
          return ex;
        }
        c[k] = cn;
        nrm[k] = nn;
        onb(nn, &u[k], &v[k]);
        In[k] = cn;
      } else {
        double aw = dot(ea, w[k]), bw = dot(eb, w[k]);
        double hw = (1.0 - aw * aw) / a + (1.0 - bw * bw) / b;
        double dt = hw > 1e-12 * (1.0 / a + 1.0 / b) ? -p.gamma * g[k][0] / hw : -eta * g[k][0];
        if (std::fabs(dt) > s.hs) dt = std::copysign(s.hs, dt);
        tpar[k] += dt;                           // D_k = c_k + t_k w_k
        In[k] = c[k] + tpar[k] * w[k];
        const Edge& E = s.edges[s.ies[cp.ie[k - 1]].edge];
        double along = dot(In[k] - E.p0, w[k]);
        if (along < 0.0 || along > elen[k]) {
          ex.status = ST_OFF_EDGE; ex.iters = it; ex.grad = gn;
          return ex;
        }
      }
    }
    for (int k = 1; k <= n; ++k) I[k] = In[k];
  }
  if (!converged) {
    gradient(n, I, cp.type, u, v, w, g);
    double g2 = 0;
    for (int k = 1; k <= n; ++k) g2 += g[k][0] * g[k][0] + g[k][1] * g[k][1];
    gn = std::sqrt(g2);
  }
  ex.iters = it;
  ex.grad = gn;
  for (int k = 1; k <= n; ++k) ex.pts[k - 1] = I[k];
  if (!(gn < p.delta)) { ex.status = ST_NOT_CONVERGED; return ex; }
  // Lastly the visibility between consecutive path nodes is validated by RT.
  for (int k = 0; k <= n; ++k) {
    Endpoint ea{IGN_NONE, NONE_LABEL}, eb{IGN_NONE, NONE_LABEL};
    if (k >= 1) ea = Endpoint{cp.type[k - 1] == T_DIFF ? IGN_ANY : IGN_LABEL, cp.label[k - 1]};
    if (k + 1 <= n) eb = Endpoint{cp.type[k] == T_DIFF ? IGN_ANY : IGN_LABEL, cp.label[k]};
    if (!visible(s, I[k], I[k + 1], ea, eb)) { ex.status = ST_OCCLUDED; return ex; }
  }
  double L = 0;
  for (int k = 0; k <= n; ++k) L += norm(I[k + 1] - I[k]);
  ex.length = L;
  ex.delay = L / C_LIGHT;
  ex.status = ST_VALID;
  return ex;
}

struct ExactSet {
  std::vector<Exact> all;     // one per coarse path, with status
  std::vector<Exact> paths;   // after duplicate removal
};

bool seq_less(const Exact& a, const Exact& b) {
  if (a.n != b.n) return a.n < b.n;
  for (int q = 0; q < a.n; ++q) {
    if (a.type[q] != b.type[q]) return a.type[q] < b.type[q];
    if (a.label[q] != b.label[q]) return a.label[q] < b.label[q];
  }
  return false;
}
bool ie_less(const Exact& a, const Exact& b) {
  for (int q = 0; q < std::min(a.n, b.n); ++q)
    if (a.ie[q] != b.ie[q]) return a.ie[q] < b.ie[q];
  return a.n < b.n;
}

// First-Fresnel-zone duplicate removal (Section 2.3) over paths already reduced to one
// per label sequence: sort by delay; a path is dropped if an earlier kept path has the
// same chain of interaction types and each of its interaction points lies within that
// path's first Fresnel zone radius r_k = sqrt(lambda a_k b_k / (a_k + b_k)), a_k and b_k
// the kept path's lengths from the TX to I_k and from I_k to the RX.  Reading for ties:
// delays are compared in bins of 1 um of length, so paths of equal length up to
// rounding are ordered by their interaction types and labels.
std::vector<Exact> fresnel_dedup(std::vector<Exact> best, const std::vector<V3>& tx, double lambda) {
  std::sort(best.begin(), best.end(), [](const Exact& a, const Exact& b) {
    if (a.tx != b.tx) return a.tx < b.tx;
    if (a.rx != b.rx) return a.rx < b.rx;
    long long qa = (long long)std::floor(a.length * 1e6), qb = (long long)std::floor(b.length * 1e6);
    if (qa != qb) return qa < qb;
    if (seq_less(a, b)) return true;
    if (seq_less(b, a)) return false;
    return ie_less(a, b);
  });
  std::vector<Exact> kept;
  for (size_t i = 0; i < best.size(); ++i) {
    const Exact& B = best[i];
    bool dup = false;
    for (const Exact& A : kept) {
      if (A.tx != B.tx || A.rx != B.rx || A.n != B.n || A.n == 0) continue;
      bool same_chain = true;
      for (int q = 0; q < A.n; ++q) same_chain = same_chain && A.type[q] == B.type[q];
      if (!same_chain) continue;
      V3 prev = tx[A.tx];
      double acc = 0.0;
      bool inside = true;
      for (int q = 0; q < A.n && inside; ++q) {
        acc += norm(A.pts[q] - prev);
        prev = A.pts[q];
        double ak = acc, bk = A.length - acc;
        double r = std::sqrt(lambda * ak * bk / (ak + bk));
        inside = norm(B.pts[q] - A.pts[q]) <= r;
      }
      if (inside) { dup = true; break; }
    }
    if (!dup) kept.push_back(B);
  }
  return kept;
}

ExactSet* refine(const Scene& s, const CoarseSet& cs) {
  ExactSet* out = new ExactSet();
  for (size_t i = 0; i < cs.paths.size(); ++i) {
    Exact e = refine_one(s, cs, cs.paths[i]);
    e.coarse = (int64_t)i;
    out->all.push_back(e);
  }
  // Label-based duplicate removal (Section 2.3): per TX/RX pair keep the shortest
  // path for each interaction-type and label combination (ties: IE sequence).
  std::vector<Exact> valid;
  for (const Exact& e : out->all)
    if (e.status == ST_VALID) valid.push_back(e);
  std::sort(valid.begin(), valid.end(), [](const Exact& a, const Exact& b) {
    if (a.tx != b.tx) return a.tx < b.tx;
    if (a.rx != b.rx) return a.rx < b.rx;
    if (seq_less(a, b)) return true;
    if (seq_less(b, a)) return false;
    if (a.length != b.length) return a.length < b.length;
    return ie_less(a, b);
  });
  std::vector<Exact> best;
  for (size_t i = 0; i < valid.size(); ++i) {
    if (i > 0 && valid[i].tx == valid[i - 1].tx && valid[i].rx == valid[i - 1].rx &&
        !seq_less(valid[i], valid[i - 1]) && !seq_less(valid[i - 1], valid[i]))
      continue;
    best.push_back(valid[i]);
  }
  out->paths = fresnel_dedup(std::move(best), cs.tx, C_LIGHT / s.p.freq_hz);
  return out;
}

}  // namespace

// =========================================================================== C interface
extern "C" {

void* oracle_voxelize(const float* xyz, const float* nrm, const uint32_t* label, const uint8_t* material,
                      int64_t n, const double* edges, const uint32_t* edge_label, int64_t n_edges,
                      const double* region, const oracle_params* p) {
  return voxelize(xyz, nrm, label, material, n, edges, edge_label, n_edges, region, p);
}

void oracle_scene_free(void* s) { delete (Scene*)s; }

// First-Fresnel-zone duplicate removal alone: m exact paths as arrays -- tx, rx, n,
// type[m][8], label[m][8], pts[m][8][3], length[m] -- with the TX positions
// tx_pos[n_tx][3] and the wavelength.  keep[m] receives 1 for each kept path.  Returns
// the number kept.
int64_t oracle_fresnel_dedup(int64_t m, const int32_t* tx, const int32_t* rx, const int32_t* n, const int32_t* type,
                             const uint32_t* label, const double* pts, const double* length, const double* tx_pos,
                             int32_t n_tx, double lambda, int32_t* keep) {
  std::vector<V3> txs;
  for (int t = 0; t < n_tx; ++t) txs.push_back(mk(tx_pos[3 * t], tx_pos[3 * t + 1], tx_pos[3 * t + 2]));
  std::vector<Exact> best;
  for (int64_t i = 0; i < m; ++i) {
    Exact e{};
    e.tx = tx[i];
    e.rx = rx[i];
    e.n = n[i];
    for (int q = 0; q < MAXI; ++q) {
      e.type[q] = type[i * MAXI + q];
      e.label[q] = label[i * MAXI + q];
      e.ie[q] = 0;
      e.pts[q] = mk(pts[(i * MAXI + q) * 3], pts[(i * MAXI + q) * 3 + 1], pts[(i * MAXI + q) * 3 + 2]);
    }
    e.length = length[i];
    e.coarse = i;
    best.push_back(e);
  }
  std::vector<Exact> kept = fresnel_dedup(std::move(best), txs, lambda);
  for (int64_t i = 0; i < m; ++i) keep[i] = 0;
  for (const Exact& e : kept) keep[e.coarse] = 1;
  return (int64_t)kept.size();
}

// Grid and table sizes: origin[3], dims[3]; returns the number of IEs.
int64_t oracle_scene_info(void* sp, double* origin, int32_t* dims, int64_t* n_points_grouped) {
  Scene* s = (Scene*)sp;
  origin[0] = s->origin.x; origin[1] = s->origin.y; origin[2] = s->origin.z;
  for (int a = 0; a < 3; ++a) dims[a] = s->dims[a];
  if (n_points_grouped) *n_points_grouped = (int64_t)s->pts.size();
  return (int64_t)s->ies.size();
}

// IE table: kind, label, cell, subvoxel coords (3), point range (2), reception point (3),
// normal (3), bbox centre (3), subvoxel centre (3), edge index, t0, t1.
void oracle_scene_ies(void* sp, int32_t* kind, uint32_t* label, int64_t* cell, int32_t* gs,
                      int64_t* prange, double* rp, double* normal, double* bbc, double* sc,
                      int32_t* edge, double* trange, uint8_t* material) {
  Scene* s = (Scene*)sp;
  for (size_t i = 0; i < s->ies.size(); ++i) {
    const IE& e = s->ies[i];
    kind[i] = e.kind; label[i] = e.label; cell[i] = e.cell;
    for (int a = 0; a < 3; ++a) {
      gs[3 * i + a] = e.gs[a];
      rp[3 * i + a] = comp(e.rp, a);
      normal[3 * i + a] = comp(e.normal, a);
      bbc[3 * i + a] = comp(e.bbc, a);
      sc[3 * i + a] = comp(e.sc, a);
    }
    prange[2 * i] = e.p_begin; prange[2 * i + 1] = e.p_count;
    edge[i] = e.edge; trange[2 * i] = e.t0; trange[2 * i + 1] = e.t1;
    material[i] = e.material;
  }
}

// Point positions and normals in the grouped order the IE point ranges index.
void oracle_scene_points(void* sp, double* xyz, double* nrm) {
  Scene* s = (Scene*)sp;
  for (size_t i = 0; i < s->pts.size(); ++i)
    for (int a = 0; a < 3; ++a) {
      xyz[3 * i + a] = comp(s->pts[i], a);
      nrm[3 * i + a] = comp(s->nrm[i], a);
    }
}

void oracle_scene_cells(void* sp, int64_t* begin, int32_t* count, int32_t* march) {
  Scene* s = (Scene*)sp;
  for (int64_t c = 0; c < s->n_cells; ++c) {
    begin[c] = s->cell_begin[c]; count[c] = s->cell_count[c]; march[c] = s->march[c];
  }
}

// Returns null when a TX or RX lies outside the voxel grid.
void* oracle_trace(void* sp, const double* tx, int32_t ntx, const double* rx, int32_t nrx) {
  const Scene& s = *(Scene*)sp;
  for (int i = 0; i < ntx + nrx; ++i) {
    const double* q = i < ntx ? tx + 3 * i : rx + 3 * (i - ntx);
    for (int a = 0; a < 3; ++a) {
      double rel = (q[a] - comp(s.origin, a)) / s.h;
      if (!(rel >= 0.0 && rel < (double)s.dims[a])) return nullptr;
    }
  }
  return trace(s, tx, ntx, rx, nrx);
}
void oracle_coarse_free(void* c) { delete (CoarseSet*)c; }

// stats: [n_paths, n_before_kappa, n_cones, n_vis, n_evals, n_levels, nodes per level...]
void oracle_coarse_stats(void* cp, int64_t* out, int32_t n_out) {
  CoarseSet* c = (CoarseSet*)cp;
  std::vector<int64_t> v = {(int64_t)c->paths.size(), c->n_before_kappa, c->n_cones, c->n_vis,
                            c->n_evals, (int64_t)c->nodes_per_level.size()};
  for (int64_t x : c->nodes_per_level) v.push_back(x);
  for (int32_t i = 0; i < n_out; ++i) out[i] = i < (int32_t)v.size() ? v[i] : 0;
}

void oracle_coarse_get(void* cp, int32_t* tx, int32_t* rx, int32_t* n, int64_t* ie, int32_t* type,
                       uint32_t* label, double* miss) {
  CoarseSet* c = (CoarseSet*)cp;
  for (size_t i = 0; i < c->paths.size(); ++i) {
    const Coarse& p = c->paths[i];
    tx[i] = p.tx; rx[i] = p.rx; n[i] = p.n; miss[i] = p.miss;
    for (int q = 0; q < MAXI; ++q) {
      ie[MAXI * i + q] = q < p.n ? p.ie[q] : -1;
      type[MAXI * i + q] = q < p.n ? p.type[q] : -1;
      label[MAXI * i + q] = q < p.n ? p.label[q] : NONE_LABEL;
    }
  }
}

void* oracle_refine(void* sp, void* cp) { return refine(*(Scene*)sp, *(CoarseSet*)cp); }

// Refine given coarse paths one by one (no duplicate removal), for sampled checks of
// another implementation's refinement: coarse path i runs from TX tx_idx[i] to RX
// rx_idx[i] through n[i] interactions (ie, type, label rows of MAXI).  Writes the
// status, iterations, final gradient norm, points (MAXI*3) and length per path.
void oracle_refine_given(void* sp, const double* tx, int32_t ntx, const double* rx, int32_t nrx, int64_t m,
                         const int32_t* tx_idx, const int32_t* rx_idx, const int32_t* n, const int64_t* ie,
                         const int32_t* type, const uint32_t* label, int32_t* status, int32_t* iters,
                         double* grad, double* pts, double* length) {
  const Scene& s = *(Scene*)sp;
  CoarseSet cs;
  for (int t = 0; t < ntx; ++t) cs.tx.push_back(mk(tx[3 * t], tx[3 * t + 1], tx[3 * t + 2]));
  for (int j = 0; j < nrx; ++j) cs.rx.push_back(mk(rx[3 * j], rx[3 * j + 1], rx[3 * j + 2]));
  for (int64_t i = 0; i < m; ++i) {
    Coarse c;
    std::memset(&c, 0, sizeof c);
    c.tx = tx_idx[i];
    c.rx = rx_idx[i];
    c.n = n[i];
    for (int q = 0; q < c.n; ++q) {
      c.ie[q] = ie[MAXI * i + q];
      c.type[q] = type[MAXI * i + q];
      c.label[q] = label[MAXI * i + q];
    }
    Exact e = refine_one(s, cs, c);
    status[i] = e.status;
    iters[i] = e.iters;
    grad[i] = e.grad;
    length[i] = e.length;
    for (int q = 0; q < MAXI; ++q)
      for (int a = 0; a < 3; ++a) pts[3 * (MAXI * i + q) + a] = q < c.n ? comp(e.pts[q], a) : 0.0;
  }
}
void oracle_exact_free(void* e) { delete (ExactSet*)e; }

// which = 0: paths after duplicate removal; 1: every refined coarse path with status.
int64_t oracle_exact_count(void* ep, int32_t which) {
  ExactSet* e = (ExactSet*)ep;
  return (int64_t)(which ? e->all.size() : e->paths.size());
}

void oracle_exact_get(void* ep, int32_t which, int32_t* tx, int32_t* rx, int32_t* n, int32_t* type,
                      uint32_t* label, uint8_t* material, int64_t* ie, double* pts, double* length,
                      double* delay, double* grad, int32_t* iters, int32_t* status, int64_t* coarse) {
  ExactSet* e = (ExactSet*)ep;
  const std::vector<Exact>& v = which ? e->all : e->paths;
  for (size_t i = 0; i < v.size(); ++i) {
    const Exact& p = v[i];
    tx[i] = p.tx; rx[i] = p.rx; n[i] = p.n; length[i] = p.length; delay[i] = p.delay;
    grad[i] = p.grad; iters[i] = p.iters; status[i] = p.status; coarse[i] = p.coarse;
    for (int q = 0; q < MAXI; ++q) {
      bool in = q < p.n;
      type[MAXI * i + q] = in ? p.type[q] : -1;
      label[MAXI * i + q] = in ? p.label[q] : NONE_LABEL;
      material[MAXI * i + q] = in ? p.material[q] : 255;
      ie[MAXI * i + q] = in ? p.ie[q] : -1;
      for (int a = 0; a < 3; ++a) pts[3 * (MAXI * i + q) + a] = in ? comp(p.pts[q], a) : 0.0;
    }
  }
}

// ------------------------------------------------------------------ building blocks (pins)
int32_t oracle_sdf(void* sp, int64_t ie, const double* x, double* f, double* n) {
  Scene* s = (Scene*)sp;
  V3 nn;
  bool ok = sdf_eval(*s, s->ies[ie], mk(x[0], x[1], x[2]), f, &nn);
  n[0] = nn.x; n[1] = nn.y; n[2] = nn.z;
  return ok ? 1 : 0;
}

int32_t oracle_sdf_label(void* sp, uint32_t label, const double* x, double* f, double* n) {
  Scene* s = (Scene*)sp;
  V3 nn;
  bool ok = sdf_label(*s, label, mk(x[0], x[1], x[2]), f, &nn);
  n[0] = nn.x; n[1] = nn.y; n[2] = nn.z;
  return ok ? 1 : 0;
}

int32_t oracle_sdf_hit(void* sp, int64_t ie, const double* P, const double* d, double* t) {
  Scene* s = (Scene*)sp;
  return sdf_hit(*s, s->ies[ie], mk(P[0], P[1], P[2]), unit(mk(d[0], d[1], d[2])), t) ? 1 : 0;
}

// Re-projection of Section 2.3 alone: the ray from P toward R met by the surface of
// label `label`; writes the new interaction point and its normal.  0 on a miss.
int32_t oracle_reproject(void* sp, const double* P, const double* R, uint32_t label, double* c, double* n) {
  V3 cn, nn;
  if (!reproject(*(Scene*)sp, mk(P[0], P[1], P[2]), mk(R[0], R[1], R[2]), label, &cn, &nn)) return 0;
  c[0] = cn.x; c[1] = cn.y; c[2] = cn.z;
  n[0] = nn.x; n[1] = nn.y; n[2] = nn.z;
  return 1;
}

// mode: 0 none, 1 same label, 2 any label near that endpoint; brute: 1 = all-voxel slab test.
int32_t oracle_visible(void* sp, const double* a, const double* b, int32_t mode_a, uint32_t label_a,
                       int32_t mode_b, uint32_t label_b, int32_t brute) {
  Scene* s = (Scene*)sp;
  Endpoint ea{mode_a, label_a}, eb{mode_b, label_b};
  V3 A = mk(a[0], a[1], a[2]), B = mk(b[0], b[1], b[2]);
  return (brute ? visible_bruteforce(*s, A, B, ea, eb) : visible(*s, A, B, ea, eb)) ? 1 : 0;
}

int32_t oracle_cone_sphere(const double* apex, const double* axis, double half_angle, const double* c,
                           double r) {
  return cone_sphere(mk(apex[0], apex[1], apex[2]), unit(mk(axis[0], axis[1], axis[2])),
                     std::sin(half_angle), std::cos(half_angle), mk(c[0], c[1], c[2]), r)
             ? 1 : 0;
}

void oracle_fibonacci(int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) fibonacci_dir(i, n, out + 3 * i);
}

void oracle_onb(const double* n, double* u, double* v) {
  V3 a, b;
  onb(mk(n[0], n[1], n[2]), &a, &b);
  u[0] = a.x; u[1] = a.y; u[2] = a.z;
  v[0] = b.x; v[1] = b.y; v[2] = b.z;
}

// Voxel cells visited by the traversal of the segment a -> b (for traversal pins).
int64_t oracle_dda_cells(void* sp, const double* a, const double* b, int64_t* out, int64_t cap) {
  Scene* s = (Scene*)sp;
  V3 A = mk(a[0], a[1], a[2]), B = mk(b[0], b[1], b[2]);
  double T = norm(B - A);
  int64_t k = 0;
  dda(*s, A, unit(B - A), T, [&](const int v[3]) {
    if (k < cap) out[k] = cell_of(*s, v[0], v[1], v[2]);
    ++k;
    return true;
  });
  return k;
}

}  // extern "C"
