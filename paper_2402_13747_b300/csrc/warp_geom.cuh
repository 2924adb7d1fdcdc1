// Warp-cooperative pieces shared by the propagation levels and the refinement:
// Eq. 1 sums split across a warp's lanes, the Section 2.2.1 march on them, and a
// visibility ray walked by the whole warp.  Every lane of the warp must call these
// together (full-mask shuffles); every lane gets the same result.  bytes is each
// lane's share of the records read (sum it over the warp).
#pragma once

#include "nimbus_internal.cuh"

namespace nb {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Warp sums of eight values, returned to every lane: a reduce-scatter (each xor
// level keeps half of the values and sends the other half, 4 + 2 + 1 shuffles), two
// more levels on the last value, then one broadcast per value -- 16 shuffles
// instead of 40 for eight independent butterflies.  After the scatter levels lane L
// holds the total of value ((L>>2)&1) + 2((L>>3)&1) + 4((L>>4)&1), i.e. value q sits
// in lane 4q.
__device__ __forceinline__ void wsum8(float v[8], int lane) {
  const bool u4 = lane & 16, u3 = lane & 8, u2 = lane & 4;
  float a[4], b[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float send = u4 ? v[k] : v[k + 4], keep = u4 ? v[k + 4] : v[k];
    a[k] = keep + __shfl_xor_sync(FULL, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float send = u3 ? a[k] : a[k + 2], keep = u3 ? a[k + 2] : a[k];
    b[k] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  float send = u2 ? b[0] : b[1], c = (u2 ? b[1] : b[0]) + __shfl_xor_sync(FULL, send, 4);
  c += __shfl_xor_sync(FULL, c, 2);
  c += __shfl_xor_sync(FULL, c, 1);
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __shfl_sync(FULL, c, 4 * k);
}

// One Eq. 1 term: point P with normal N (both relative to the frame of x) adds its
// Gaussian weight to the sums (weight, weighted position, weighted normal).
__device__ __forceinline__ void eq1_term(float v[8], float3 x, float4 P, float4 N, float3 c, float inv_s2) {
  float3 p = xyz(P) - c;
  float3 d = x - p;
  float w = expf(-dot(d, d) * inv_s2);
  v[0] += w;
  v[1] += w * p.x; v[2] += w * p.y; v[3] += w * p.z;
  v[4] += w * N.x; v[5] += w * N.y; v[6] += w * N.z;
}

// f and normal from the reduced sums; false when every weight vanished.
__device__ __forceinline__ bool eq1_finish(const float v[8], float3 x, float* f, float3* n_out) {
  if (!(v[0] > 0.f)) return false;
  float3 sn = f3(v[4], v[5], v[6]);
  float nn = len(sn);
  if (!(nn > 0.f)) return false;
  float3 n = (1.f / nn) * sn;
  float3 p = (1.f / v[0]) * f3(v[1], v[2], v[3]);
  *f = dot(x - p, n);
  if (n_out) *n_out = n;
  return true;
}

// Eq. 1 over the points of one IE, the points split across the warp's lanes; every
// lane returns the same f and normal.  c is the IE's bounding-box centre, x is
// relative to c.
// Lane l adds points l, l + 32, l + 64, ... in that order.  With NB_VIS_PAIRS (the
// default) each pass loads two of them before adding either, so two loads are in
// flight per lane (an IE of the 3 cm scans holds about 70 points: two passes instead
// of three); the order of the sums is the same either way.  A translation unit may
// set it to 0 before including this header (the refinement does: its kernel's code
// was measured faster so, with the final visibility rays a negligible share of it).
#ifndef NB_VIS_PAIRS
#define NB_VIS_PAIRS 1
#endif
__device__ bool sdf_warp(const DScene& s, uint32_t pb, uint32_t pc, float3 c, float3 x, float* f, float3* n_out,
                         int lane, unsigned long long& bytes) {
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#if NB_VIS_PAIRS
  for (uint32_t k = lane; k < pc; k += 64) {
    const uint32_t k1 = k + 32 < pc ? k + 32 : k;   // past the end: re-read point k, unused
    const float4 P0 = __ldg(&s.pts[pb + k]), N0 = __ldg(&s.pnrm[pb + k]);
    const float4 P1 = __ldg(&s.pts[pb + k1]), N1 = __ldg(&s.pnrm[pb + k1]);
    eq1_term(v, x, P0, N0, c, s.sdf_inv_s2);
    if (k + 32 < pc) eq1_term(v, x, P1, N1, c, s.sdf_inv_s2);
  }
#else
  for (uint32_t k = lane; k < pc; k += 32) eq1_term(v, x, __ldg(&s.pts[pb + k]), __ldg(&s.pnrm[pb + k]), c, s.sdf_inv_s2);
#endif
  if (lane == 0) bytes += 24ull * pc;
  wsum8(v, lane);
  return eq1_finish(v, x, f, n_out);
}

// The Eq. 1 march of Section 2.2.1 (see sdf_march) with warp-shared sums.
__device__ bool sdf_march_warp(const DScene& s, uint32_t pb, uint32_t pc, float3 c, float3 x0, float3 d,
                               float* tau_hit, int lane, unsigned long long& bytes) {
  const float half = 0.5f * s.seg_len;
  auto eval = [&](float t, float* f, float3* n) { return sdf_warp(s, pb, pc, c, x0 + t * d, f, n, lane, bytes); };
  return march_abs_f<true>(eval, d, -half, half, s.sdf_eps, s.sdf_max_steps, tau_hit);
}

// Visibility ray A -> B (Section 2.3's final check) with the warp: the walk is shared,
// the IEs of each voxel are screened by the lanes, candidates are marched together.
__device__ bool visible_warp(const DScene& s, float3 A, float3 B, Endpoint ea, Endpoint eb, int lane,
                             unsigned long long& bytes) {
  float3 dv = B - A;
  float T = len(dv);
  if (T < 1e-9f) return true;
  float3 d = (1.f / T) * dv;
  Walk w;
  walk_init(s, A, d, w);
  const int max_steps = s.nx + s.ny + s.nz + 3;
  for (int step = 0; step < max_steps; ++step) {
    uint2 cell = __ldg(&s.cells[cell_index(s, w.v[0], w.v[1], w.v[2])]);
    for (uint32_t base = 0; base < cell.y; base += 32) {
      // each lane screens one IE of the voxel: its sphere against the segment, then
      // the two exact march skips (cannot occlude, cannot hit), so that the warp walks
      // the IEs one by one only for the marches that must run
      const uint32_t k = base + lane;
      const uint32_t id = cell.x + k;
      bool ok = false;
      if (k < cell.y) {
        const IERec* r = &s.ies[id];
        const float4 sc = __ldg(&r->sc_pc);
        const float4 nm = __ldg(&r->nrm_meta);
        bytes += 32;
        ok = (__float_as_uint(nm.w) & 1u) == IE_POINT && segment_sphere(A, d, T, xyz(sc), s.r_sub);
        if (ok) {
          const float3 c = xyz(__ldg(&r->bbc_pb));
          const float tc = dot(c - A, d);
          const uint32_t lbl = __float_as_uint(__ldg(&r->rp_lab).w);
          ok = !cannot_occlude(ea, eb, lbl, tc, 0.5f * s.seg_len, T, s.vis_ignore);
          if (ok) {
            bytes += 32;
            ok = !march_cannot_hit(__ldg(&r->slab), xyz(nm), (A - c) + tc * d, d, 0.5f * s.seg_len, s.sdf_eps);
          }
        }
      }
      unsigned mask = __ballot_sync(FULL, ok);
      while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        const IERec* r = &s.ies[__shfl_sync(FULL, id, j)];
        const float4 bb = __ldg(&r->bbc_pb);
        const float4 sc = __ldg(&r->sc_pc);
        const float3 c = xyz(bb);
        const float tc = dot(c - A, d);
        const uint32_t lj = __float_as_uint(__ldg(&r->rp_lab).w);
        const float3 xj = (A - c) + tc * d;
        float tau;
        if (!sdf_march_warp(s, __float_as_uint(bb.w), __float_as_uint(sc.w), c, xj, d, &tau, lane, bytes)) continue;
        const float th = tc + tau;
        if (!(th > 0.f && th < T)) continue;
        if (ignored(ea, lj, th, s.vis_ignore) || ignored(eb, lj, T - th, s.vis_ignore)) continue;
        return false;
      }
    }
    if (!walk_next(s, w, T)) break;
  }
  return true;
}

}  // namespace
}  // namespace nb
