// Prefix sums and a stable least-significant-digit radix sort.
//
// Sorting by key is the core of voxelisation (points grouped per subvoxel and
// label, Section 2.1) and of the duplicate limit and duplicate removal steps
// (Sections 2.2.3, 2.3).  The sort is a plain three-kernel LSD pass per 8-bit
// digit: per-tile digit histograms, one exclusive scan over the digit-major
// histogram table, and a stable scatter whose in-tile ranks come from warp
// match masks, so equal keys keep their input order.
#include <cstdio>

#include "nimbus_host.hpp"

namespace nb {

namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

constexpr int RS_BLOCK = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RS_RADIX = 256;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Per-tile exclusive scan; writes the tile sum to block_sums (if not null).
__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t s_warp[SCAN_BLOCK / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0u;
    sum += v[i];
  }
  uint32_t incl = warp_incl_scan(sum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < SCAN_BLOCK / 32 ? s_warp[lane] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (lane < SCAN_BLOCK / 32) s_warp[lane] = wi - w;
  }
  __syncthreads();
  uint32_t run = s_warp[warp] + incl - sum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
  if (block_sums && threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ offs) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const uint32_t add = offs[blockIdx.x];
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_BLOCK) {
    int64_t idx = base + i;
    if (idx < n) out[idx] += add;
  }
}

__global__ void k_total(const uint32_t* in_last, const uint32_t* out_last, uint32_t* total) {
  *total = *in_last + *out_last;
}

int scan_rec(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n) {
  if (n <= 0) return NIMBUS_OK;
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    k_scan_tiles<<<1, SCAN_BLOCK, 0, sc.st>>>(in, out, n, nullptr);
    NB_LAUNCHED(sc.mem->err);
    return NIMBUS_OK;
  }
  uint32_t* sums;
  uint32_t* sums_scanned;
  NB_TRY(sc.get(&sums, nb));
  NB_TRY(sc.get(&sums_scanned, nb));
  k_scan_tiles<<<(unsigned)nb, SCAN_BLOCK, 0, sc.st>>>(in, out, n, sums);
  NB_LAUNCHED(sc.mem->err);
  NB_TRY(scan_rec(sc, sums, sums_scanned, nb));
  k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, sc.st>>>(out, n, sums_scanned);
  NB_LAUNCHED(sc.mem->err);
  return NIMBUS_OK;
}

// Digit histogram of one tile, written digit-major: hist[d * n_tiles + tile].
__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                          int64_t n_tiles) {
  __shared__ uint32_t s_h[RS_RADIX];
  for (int i = threadIdx.x; i < RS_RADIX; i += RS_BLOCK) s_h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_BLOCK) {
    int64_t idx = base + i;
    if (idx < n) atomicAdd(&s_h[(keys[idx] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_RADIX; d += RS_BLOCK) hist[(int64_t)d * n_tiles + blockIdx.x] = s_h[d];
}

// Stable scatter of one tile.  Items are visited in index order (RS_ITEMS rounds of
// one item per thread, thread order inside a round); the rank of an item among
// equal digits is the running count of earlier rounds, plus the counts of earlier
// warps in this round, plus its rank inside its warp (match mask).
__global__ void k_rs_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                             uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n,
                             int shift, const uint32_t* __restrict__ offs, int64_t n_tiles) {
  __shared__ uint32_t s_base[RS_RADIX];
  __shared__ uint32_t s_run[RS_RADIX];
  __shared__ uint32_t s_wc[RS_WARPS][RS_RADIX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < RS_RADIX; d += RS_BLOCK) {
    s_base[d] = offs[(int64_t)d * n_tiles + blockIdx.x];
    s_run[d] = 0;
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    for (int i = threadIdx.x; i < RS_WARPS * RS_RADIX; i += RS_BLOCK) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    int64_t idx = base + (int64_t)r * RS_BLOCK + threadIdx.x;
    bool valid = idx < n;
    uint64_t k = valid ? keys[idx] : 0ull;
    uint32_t d = valid ? (uint32_t)((k >> shift) & 0xffu) : 0x100u;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t lrank = __popc(peers & lt_mask);
    if (valid && lrank == 0) s_wc[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pre = s_run[d];
      for (int w2 = 0; w2 < warp; ++w2) pre += s_wc[w2][d];
      uint32_t pos = s_base[d] + pre + lrank;
      keys_out[pos] = k;
      vals_out[pos] = vals[idx];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < RS_RADIX; dd += RS_BLOCK) {
      uint32_t add = 0;
      for (int w2 = 0; w2 < RS_WARPS; ++w2) add += s_wc[w2][dd];
      s_run[dd] += add;
    }
    __syncthreads();
  }
}

}  // namespace

int exclusive_scan(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total) {
  if (n <= 0) {
    if (total) NB_CUDA(sc.mem->err, cudaMemsetAsync(total, 0, sizeof(uint32_t), sc.st));
    return NIMBUS_OK;
  }
  // the total needs the last input, which an in-place scan would overwrite
  uint32_t* last_in = nullptr;
  if (total) {
    NB_TRY(sc.get(&last_in, 1));
    NB_CUDA(sc.mem->err, cudaMemcpyAsync(last_in, in + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToDevice, sc.st));
  }
  NB_TRY(scan_rec(sc, in, out, n));
  if (total) {
    k_total<<<1, 1, 0, sc.st>>>(last_in, out + (n - 1), total);
    NB_LAUNCHED(sc.mem->err);
  }
  return NIMBUS_OK;
}

// The gets of scan_rec, level by level.
static size_t scan_rec_arena_bytes(int64_t n) {
  size_t b = 0;
  while (n > 0) {
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) break;
    b += 2 * Scratch::arena_block((size_t)nb, sizeof(uint32_t));
    n = nb;
  }
  return b;
}

size_t scan_arena_bytes(int64_t n, bool total) {
  if (n <= 0) return 0;
  return (total ? Scratch::arena_block(1, sizeof(uint32_t)) : 0) + scan_rec_arena_bytes(n);
}

size_t radix_arena_bytes(int64_t n, int bits) {
  if (n <= 1 || bits <= 0) return 0;
  const int64_t n_tiles = (n + RS_TILE - 1) / RS_TILE;
  const int passes = (bits + 7) / 8;
  return 2 * Scratch::arena_block((size_t)RS_RADIX * n_tiles, sizeof(uint32_t)) +
         (size_t)passes * scan_arena_bytes((int64_t)RS_RADIX * n_tiles, false);
}

int radix_sort(Scratch& sc, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
               int bits) {
  if (n <= 1 || bits <= 0) return NIMBUS_OK;
  int64_t n_tiles = (n + RS_TILE - 1) / RS_TILE;
  uint32_t* hist;
  uint32_t* offs;
  NB_TRY(sc.get(&hist, (size_t)RS_RADIX * n_tiles));
  NB_TRY(sc.get(&offs, (size_t)RS_RADIX * n_tiles));
  uint64_t* kin = keys;
  uint32_t* vin = vals;
  uint64_t* kout = keys_alt;
  uint32_t* vout = vals_alt;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_rs_hist<<<(unsigned)n_tiles, RS_BLOCK, 0, sc.st>>>(kin, n, shift, hist, n_tiles);
    NB_LAUNCHED(sc.mem->err);
    NB_TRY(exclusive_scan(sc, hist, offs, (int64_t)RS_RADIX * n_tiles, nullptr));
    k_rs_scatter<<<(unsigned)n_tiles, RS_BLOCK, 0, sc.st>>>(kin, vin, kout, vout, n, shift, offs, n_tiles);
    NB_LAUNCHED(sc.mem->err);
    uint64_t* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
  if (kin != keys) {
    NB_CUDA(sc.mem->err, cudaMemcpyAsync(keys, kin, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, sc.st));
    NB_CUDA(sc.mem->err, cudaMemcpyAsync(vals, vin, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, sc.st));
  }
  return NIMBUS_OK;
}

}  // namespace nb
