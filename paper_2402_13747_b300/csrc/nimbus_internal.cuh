// Internal device records and device functions of the CUDA library.
// Paper: "A Ray Launching Approach for Computing Exact Paths with Point Clouds"
// (arXiv 2402.13747).  Layouts are chosen for B300 (sm_103a): 16-byte records read
// with one vector load, structure-of-arrays node buffers, FP32 traversal and FP64
// only where refinement needs it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nimbus.h"

#define NB_MAXI NIMBUS_MAX_INTERACTIONS
#define NB_NONE_LABEL 0xFFFFFFFFu

namespace nb {

// ----------------------------------------------------------------------------- records
// One intersectable entity (Section 2.1), 80 bytes = five 16-byte vector loads.
//   rp_lab : ray reception point xyz, label (bits)
//   nrm_meta: mean normal xyz (point IE), meta bits: kind (bit 0), material << 8
//   bbc_pb : bounding-box centre of the points xyz, first point (point IE) or edge index
//   sc_pc  : subvoxel centre xyz, number of points
//   slab   : (point IE) bounds of its points for march_cannot_hit: the smallest cosine
//            between a point's normal and the mean normal, the smallest and largest
//            offset of a point from the bbox centre along the mean normal, and the
//            largest distance of a point from that centre; zeros for an edge
struct __align__(16) IERec {
  float4 rp_lab;
  float4 nrm_meta;
  float4 bbc_pb;
  float4 sc_pc;
  float4 slab;
};

enum { IE_POINT = 0, IE_EDGE = 1 };
enum { T_REFL = 0, T_DIFF = 1 };
enum { ST_VALID = 0, ST_MISS = 1, ST_NOT_CONVERGED = 2, ST_OCCLUDED = 3, ST_OFF_EDGE = 4 };
// endpoint self-hit rule of a visibility ray
enum { IGN_NONE = 0, IGN_LABEL = 1, IGN_ANY = 2 };

// Scene as the kernels see it (passed by value).
struct DScene {
  float ox, oy, oz;        // grid origin
  float h, inv_h, hs;      // voxel edge, its inverse, subvoxel edge
  float inv_hs;             // 1 / subvoxel edge (FP32 binning of continuous points in refinement)
  int nx, ny, nz, dv;
  double odx, ody, odz, hd, hsd;
  long long n_cells;
  int n_ie, n_edges;
  float r_vox, r_sub, seg_len;   // voxel sphere, subvoxel sphere, subvoxel diameter
  float sdf_inv_s2, sdf_eps, vis_ignore;
  int sdf_max_steps;
  const uint2* cells;      // per voxel: first IE, IE count
  const uint8_t* march;    // per voxel: capped L-inf distance to a voxel with IEs
  const IERec* ies;
  const float4* pts;       // grouped by IE: xyz, and w = the point's index in the input cloud (bits)
  const float4* pnrm;      // grouped by IE: normal xyz, unused
  const double* edges;     // [n_edges*12] p0 p1 n0 n1
};

// ----------------------------------------------------------------------------- float3 math
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }
__device__ __forceinline__ float len(float3 a) { return sqrtf(dot(a, a)); }
__device__ __forceinline__ float3 normalize(float3 a) {
  float n = sqrtf(dot(a, a));
  return n > 0.f ? (1.f / n) * a : a;
}
__device__ __forceinline__ float comp(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 D3(double x, double y, double z) { d3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return D3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return D3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return D3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double len(d3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ d3 normalize(d3 a) {
  double n = sqrt(dot(a, a));
  return n > 0.0 ? (1.0 / n) * a : a;
}
__device__ __forceinline__ float3 tof(d3 a) { return f3((float)a.x, (float)a.y, (float)a.z); }
__device__ __forceinline__ d3 tod(float3 a) { return D3(a.x, a.y, a.z); }

__device__ __forceinline__ uint32_t fbits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ float bitsf(uint32_t v) { return __uint_as_float(v); }

// Orthonormal completion (u, v) of a unit vector n: Duff et al., "Building an
// Orthonormal Basis, Revisited" (2017), in FP32 and FP64.
__device__ __forceinline__ void onb(float3 n, float3* u, float3* v) {
  float sign = copysignf(1.f, n.z);
  float a = -1.f / (sign + n.z);
  float b = n.x * n.y * a;
  *u = f3(1.f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *v = f3(b, sign + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ void onb(d3 n, d3* u, d3* v) {
  double sign = copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *u = D3(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *v = D3(b, sign + n.y * n.y * a, -n.y);
}

// ----------------------------------------------------------------------------- grid
__device__ __forceinline__ long long cell_index(const DScene& s, int x, int y, int z) {
  return ((long long)z * s.ny + y) * s.nx + x;
}
__device__ __forceinline__ bool in_grid(const DScene& s, int x, int y, int z) {
  return (unsigned)x < (unsigned)s.nx && (unsigned)y < (unsigned)s.ny && (unsigned)z < (unsigned)s.nz;
}
__device__ __forceinline__ float3 voxel_center(const DScene& s, int x, int y, int z) {
  return f3(s.ox + ((float)x + 0.5f) * s.h, s.oy + ((float)y + 0.5f) * s.h, s.oz + ((float)z + 0.5f) * s.h);
}

// Subvoxel of a position (Section 2.1) with explicitly rounded FP32 operations:
// (x - o) and then / h_s, each correctly rounded, then floor; never contracted, so
// any IEEE implementation that does the same bins every point identically.
__device__ __forceinline__ int subvoxel_axis(float x, float o, float hs, int hi) {
  float t = __fdiv_rn(__fsub_rn(x, o), hs);
  float f = floorf(t);
  return f < 0.f ? 0 : (f > (float)hi ? hi : (int)f);
}

// ----------------------------------------------------------------------------- traversal
// Amanatides-Woo voxel walk of P + t d; ties pick the lowest axis.
struct Walk {
  int v[3], step[3];
  float tmax[3], tdelta[3];
};

__device__ __forceinline__ bool walk_init(const DScene& s, float3 P, float3 d, Walk& w) {
  const float o[3] = {s.ox, s.oy, s.oz};
  const int dims[3] = {s.nx, s.ny, s.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float pa = comp(P, a), da = comp(d, a);
    int v = (int)floorf((pa - o[a]) * s.inv_h);
    v = v < 0 ? 0 : (v >= dims[a] ? dims[a] - 1 : v);
    w.v[a] = v;
    if (da > 0.f) {
      w.step[a] = 1;
      w.tmax[a] = (o[a] + (float)(v + 1) * s.h - pa) / da;
      w.tdelta[a] = s.h / da;
    } else if (da < 0.f) {
      w.step[a] = -1;
      w.tmax[a] = (o[a] + (float)v * s.h - pa) / da;
      w.tdelta[a] = -s.h / da;
    } else {
      w.step[a] = 0;
      w.tmax[a] = __int_as_float(0x7f800000);
      w.tdelta[a] = __int_as_float(0x7f800000);
    }
  }
  return true;
}

// Advance to the next voxel; false when the walk leaves the grid or passes t_end.
__device__ __forceinline__ bool walk_next(const DScene& s, Walk& w, float t_end) {
  int a = 0;
  if (w.tmax[1] < w.tmax[a]) a = 1;
  if (w.tmax[2] < w.tmax[a]) a = 2;
  if (w.tmax[a] > t_end) return false;
  w.v[a] += w.step[a];
  const int dims[3] = {s.nx, s.ny, s.nz};
  if ((unsigned)w.v[a] >= (unsigned)dims[a]) return false;
  w.tmax[a] += w.tdelta[a];
  return true;
}

// ----------------------------------------------------------------------------- cones
// Sphere (C, r) against the one-sided cone (apex A, unit axis, half-angle alpha):
// the angle between the axis and C - A may exceed alpha by at most asin(r/|C - A|).
__device__ __forceinline__ bool cone_sphere(float3 A, float3 axis, float sin_a, float cos_a, float3 C, float r) {
  float3 v = C - A;
  float d2 = dot(v, v);
  float r2 = r * r;
  if (d2 <= r2) return true;
  float t = dot(v, axis);
  return t + r * sin_a >= cos_a * sqrtf(d2 - r2);
}

__device__ __forceinline__ bool segment_sphere(float3 A, float3 d, float T, float3 C, float r) {
  float tc = fminf(fmaxf(dot(C - A, d), 0.f), T);
  float3 q = A + tc * d - C;
  return dot(q, q) <= r * r;
}

// ----------------------------------------------------------------------------- Eq. 1
// f(x) = (x - p(x)) . n(x) over the points of one IE with Gaussian weights
// exp(-|x - p_i|^2 / sigma^2).  x and the points are taken relative to the IE's
// bounding-box centre c so the FP32 sums stay well conditioned.
__device__ __forceinline__ bool sdf_local(const DScene& s, uint32_t pb, uint32_t pc, float3 c, float3 x,
                                          float* f, float3* n_out, unsigned long long& bytes) {
  bytes += 24ull * pc;
  float sw = 0.f;
  float3 sp = f3(0.f, 0.f, 0.f), sn = f3(0.f, 0.f, 0.f);
  for (uint32_t k = 0; k < pc; ++k) {
    float4 P = __ldg(&s.pts[pb + k]);
    float4 N = __ldg(&s.pnrm[pb + k]);
    float3 p = xyz(P) - c;
    float3 d = x - p;
    float w = expf(-dot(d, d) * s.sdf_inv_s2);
    sw += w;
    sp = sp + w * p;
    sn = sn + w * xyz(N);
  }
  if (!(sw > 0.f)) return false;
  float nn = len(sn);
  if (!(nn > 0.f)) return false;
  float3 n = (1.f / nn) * sn;
  float3 p = (1.f / sw) * sp;
  *f = dot(x - p, n);
  if (n_out) *n_out = n;
  return true;
}

// The |f| march of Section 2.2.1 on [t0, t_end] along unit direction d, for any
// evaluator eval(t, &f, &n) of Eq. 1 on the ray.  Steps t += |f(t)| until the sign
// of f changes (secant placement) or |f| < eps (one Newton step along the ray);
// false when the segment end is passed, the step budget runs out, every weight
// vanishes, or the Newton placement falls off the segment (the intersection lies on
// the marched segment), so a hit always satisfies t0 <= t_hit <= t_end.
// With Jump set (visibility only, where the caller keeps a yes/no decision): where
// f falls geometrically between two steps (as it does exactly on a surface that is
// linear along the ray), the step k at which the march would first see |f| < eps,
// and its position, follow in closed form; the march jumps there only if that step
// is within the budget and the segment and one evaluation there confirms |f| < eps
// with the same sign, else it continues step by step.  The placed hit then moves by
// up to eps along the ray, so the re-projection of the refinement, whose points are
// results, marches without it.
template <bool Jump, class Eval>
__device__ __forceinline__ bool march_abs_f(Eval&& eval, float3 d, float t0, float t_end, float eps, int max_steps,
                                            float* t_hit) {
  float t = t0, f;
  float3 n;
  if (!eval(t, &f, &n)) return false;
  for (int it = 0; it < max_steps; ++it) {
    if (fabsf(f) < eps) {
      float dn = dot(n, d);
      const float th = fabsf(dn) > 1e-3f ? t - f / dn : t;
      if (!(th >= t0 && th <= t_end)) return false;   // the intersection lies on the segment
      *t_hit = th;
      return true;
    }
    float tn = t + fabsf(f);
    if (tn > t_end) return false;
    float fn;
    float3 nn;
    if (!eval(tn, &fn, &nn)) return false;
    if ((fn < 0.f) != (f < 0.f)) {
      *t_hit = t - f * (tn - t) / (fn - f);
      return true;
    }
    const float a0 = fabsf(f), a1 = fabsf(fn);
    if (Jump && a1 >= eps && a1 < 0.9f * a0) {
      const float lq = __logf(a1 / a0);                      // log of the ratio, < 0
      const int k = (int)ceilf(__logf(eps / a1) / lq);        // steps after tn to |f| < eps
      if (k >= 2 && it + 1 + k < max_steps) {
        const float tk = tn + a1 * (1.f - __expf((float)k * lq)) / (1.f - a1 / a0);
        float fk;
        float3 nk;
        if (tk <= t_end && eval(tk, &fk, &nk) && fabsf(fk) < eps && ((fk < 0.f) == (fn < 0.f))) {
          t = tk;
          f = fk;
          n = nk;
          it += k;
          continue;
        }
      }
    }
    t = tn;
    f = fn;
    n = nn;
  }
  return false;
}

// Ray / point-set intersection (Section 2.2.1) in the IE's local frame for the
// visibility test: c is the IE's bounding-box centre, x0 the ray point nearest it
// (relative to c), d the unit direction; the segment [-L/2, L/2] around x0 is
// marched from its near end.  Returns the hit offset tau from x0, false on a miss.
__device__ __forceinline__ bool sdf_march(const DScene& s, uint32_t pb, uint32_t pc, float3 c, float3 x0,
                                          float3 d, float* tau_hit, unsigned long long& bytes) {
  const float half = 0.5f * s.seg_len;
  auto eval = [&](float t, float* f, float3* n) { return sdf_local(s, pb, pc, c, x0 + t * d, f, n, bytes); };
  return march_abs_f<true>(eval, d, -half, half, s.sdf_eps, s.sdf_max_steps, tau_hit);
}

struct Endpoint {
  int mode;
  uint32_t label;
};

__device__ __forceinline__ bool ignored(Endpoint e, uint32_t lbl, float dist, float r) {
  if (dist >= r) return false;
  if (e.mode == IGN_ANY) return true;
  if (e.mode == IGN_LABEL) return lbl == e.label;
  return false;
}

// True when no hit on an IE of label lbl, centred at tc along the ray of length T,
// can occlude: every hit lies on the IE's marched segment [tc - half, tc + half], and
// an endpoint whose rule ignores lbl covers that whole segment within r.  Exact in
// FP32 too: th = tc + tau with |tau| <= half gives th <= tc + half (rounding is
// monotonic), and likewise for T - th.  Skipping such an IE's march changes no
// visibility decision.
__device__ __forceinline__ bool cannot_occlude(Endpoint ea, Endpoint eb, uint32_t lbl, float tc, float half, float T,
                                               float r) {
  const bool a_ign = ea.mode == IGN_ANY || (ea.mode == IGN_LABEL && lbl == ea.label);
  const bool b_ign = eb.mode == IGN_ANY || (eb.mode == IGN_LABEL && lbl == eb.label);
  return (a_ign && tc + half < r) || (b_ign && T - (tc - half) < r);
}

// True when the march of Section 2.2.1 over an IE's Eq. 1 surface is known to miss
// the segment x0 + t d, |t| <= half (IE frame, origin at the bbox centre), without
// running it.  Eq. 1's normal is a normalised positive combination of the point
// normals, so it lies in the cone of half-angle theta around the mean normal n0
// (cos theta = slab.x); its point term is a convex combination of the points, whose
// offsets along n0 lie in [slab.y, slab.z] and whose distance from the centre is at
// most slab.w.  With that normal written cos(phi) n0 + sin(phi) u (phi <= theta, u a
// unit vector normal to n0), f(x) >= cos(theta) (x.n0 - slab.z) - sin(theta)
// (|x| + slab.w) wherever x.n0 > slab.z, and symmetrically below the slab.  x.n0 is
// linear and |x| convex along the segment, so both take their extremes at its ends.
// Where the bound keeps |f| above eps plus 1e-5 m (the FP32 rounding of f and of the
// bound is below 1e-6 m at these sizes) every evaluation the march makes has the same
// sign and |f| >= eps: it returns no hit, and skipping it changes no decision.
__device__ __forceinline__ bool march_cannot_hit(float4 slab, float3 n0, float3 x0, float3 d, float half,
                                                 float eps) {
  const float cmin = slab.x;
  if (!(cmin > 0.5f)) return false;
  const float s0 = dot(x0, n0), sd = half * fabsf(dot(d, n0));
  const float D = fmaxf(len(x0 - half * d), len(x0 + half * d)) + slab.w;
  const float need = eps + 1e-5f + sqrtf(fmaxf(0.f, 1.f - cmin * cmin)) * D;
  return (s0 - sd - slab.z) * cmin > need || (slab.y - (s0 + sd)) * cmin > need;
}

// Visibility ray A -> B (Sections 2.2.4, 2.3): walk the voxels of the segment and
// intersect the point IEs of each voxel passed.  bytes counts the scene records read.
static __device__ __noinline__ bool visible(const DScene& s, float3 A, float3 B, Endpoint ea, Endpoint eb, unsigned long long& bytes) {
  float3 dv = B - A;
  float T = len(dv);
  if (T < 1e-9f) return true;
  float3 d = (1.f / T) * dv;
  Walk w;
  walk_init(s, A, d, w);
  const int max_steps = s.nx + s.ny + s.nz + 3;
  for (int step = 0; step < max_steps; ++step) {
    uint2 cell = __ldg(&s.cells[cell_index(s, w.v[0], w.v[1], w.v[2])]);
    bytes += 8;
    for (uint32_t k = 0; k < cell.y; ++k) {
      const IERec* ie = &s.ies[cell.x + k];
      float4 sc_pc = __ldg(&ie->sc_pc);
      bytes += 16;
      if (!segment_sphere(A, d, T, xyz(sc_pc), s.r_sub)) continue;
      float4 nm = __ldg(&ie->nrm_meta);
      float4 bb = __ldg(&ie->bbc_pb);
      bytes += 32;
      if ((__float_as_uint(nm.w) & 1u) != IE_POINT) continue;   // edges never occlude
      float3 c = xyz(bb);
      float tc = dot(c - A, d);
      uint32_t lbl = __float_as_uint(__ldg(&ie->rp_lab).w);
      bytes += 16;
      if (cannot_occlude(ea, eb, lbl, tc, 0.5f * s.seg_len, T, s.vis_ignore)) continue;
      float3 x0 = (A - c) + tc * d;
      bytes += 16;
      if (march_cannot_hit(__ldg(&ie->slab), xyz(nm), x0, d, 0.5f * s.seg_len, s.sdf_eps)) continue;
      float tau;
      if (!sdf_march(s, __float_as_uint(bb.w), __float_as_uint(sc_pc.w), c, x0, d, &tau, bytes)) continue;
      float th = tc + tau;
      if (!(th > 0.f && th < T)) continue;
      if (ignored(ea, lbl, th, s.vis_ignore) || ignored(eb, lbl, T - th, s.vis_ignore)) continue;
      return false;
    }
    if (!walk_next(s, w, T)) break;
  }
  return true;
}

}  // namespace nb
