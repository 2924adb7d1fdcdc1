// C ABI of the library (include/nimbus.h): contexts, handles, the device-memory
// budget, argument checks and the copy-out of results.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "nimbus_host.hpp"

struct nimbus_ctx {
  int device = 0;
  nb::Mem mem;
  nb::GraphCache graphs;
  nb::Tuning tune;
  std::string err;
  std::unordered_map<uint64_t, nb::Obj*> objs;
  std::unordered_map<uint64_t, cudaStream_t> obj_stream;
  uint64_t next = 1;
};

namespace nb {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};

int cuda_fail(std::string* err, cudaError_t e, const char* what) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  if (err) *err = buf;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? NIMBUS_ERR_OOM : NIMBUS_ERR_CUDA;
}

int num_sms() {
  int d = 0, n = 148;
  cudaGetDevice(&d);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
  return n;
}

int Mem::alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (used + bytes > budget) {
    if (err) *err = "device memory budget exhausted";
    return NIMBUS_ERR_OOM;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(err, e, "cudaMallocAsync");
  }
  g_allocs.fetch_add(1);
  sizes[*p] = bytes;
  used += bytes;
  peak = std::max(peak, used);
  return NIMBUS_OK;
}

void Mem::release(void* p, cudaStream_t st) {
  if (!p) return;
  auto it = sizes.find(p);
  if (it == sizes.end()) return;
  used -= it->second;
  sizes.erase(it);
  cudaFreeAsync(p, st);
}

namespace {

__global__ void k_gather_exact(const ExactRec* all, const uint32_t* idx, int64_t n, ExactRec* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = all[idx[i]];
}

}  // namespace
}  // namespace nb

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <class T>
T* get_obj(nimbus_ctx* ctx, nimbus_handle h, int kind) {
  auto it = ctx->objs.find(h);
  if (it == ctx->objs.end() || it->second->kind != kind) {
    ctx->err = "unknown handle or handle of the wrong kind";
    return nullptr;
  }
  return static_cast<T*>(it->second);
}

nimbus_handle put_obj(nimbus_ctx* ctx, nb::Obj* o, cudaStream_t st) {
  nimbus_handle h = ctx->next++;
  ctx->objs[h] = o;
  ctx->obj_stream[h] = st;
  return h;
}

void drop_obj(nimbus_ctx* ctx, nb::Obj* o, cudaStream_t st) {
  o->free_all(st);
  if (o->kind == nb::OBJ_SCENE) {
    auto* s = static_cast<nb::SceneObj*>(o);
    for (void* p : s->table_bufs) ctx->mem.release(p, st);
    s->table_bufs.clear();
  }
  delete o;
}

}  // namespace

extern "C" {

int nimbus_create(nimbus_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return NIMBUS_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return NIMBUS_ERR_ARG;
  }
  nimbus_ctx* ctx = new nimbus_ctx();
  ctx->device = device;
  ctx->mem.err = &ctx->err;
  ctx->mem.graphs = &ctx->graphs;
  DeviceGuard g(device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return NIMBUS_ERR_CUDA;
  }
  ctx->mem.budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * (double)free_b);
  *out = ctx;
  return NIMBUS_OK;
}

int nimbus_destroy(nimbus_ctx* ctx) {
  if (!ctx) return NIMBUS_ERR_ARG;
  {
    DeviceGuard g(ctx->device);
    for (auto& kv : ctx->objs) drop_obj(ctx, kv.second, ctx->obj_stream[kv.first]);
    ctx->objs.clear();
    cudaDeviceSynchronize();
    ctx->graphs.release();
    cudaGetLastError();
  }
  delete ctx;
  return NIMBUS_OK;
}

const char* nimbus_last_error(nimbus_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int nimbus_voxelize(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_edges* edges,
                    const nimbus_vox_params* params, nimbus_handle* scene_out, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!scene_out || !params) {
    ctx->err = "voxelize: null argument";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  auto* S = new nb::SceneObj();
  S->mem = &ctx->mem;
  int rc = nb::voxelize_scene(ctx->mem, cloud, edges, params, S, st);
  if (rc != NIMBUS_OK) {
    drop_obj(ctx, S, st);
    return rc;
  }
  *scene_out = put_obj(ctx, S, st);
  return NIMBUS_OK;
}

int nimbus_update_region(nimbus_ctx* ctx, nimbus_handle scene, const double aabb_min[3], const double aabb_max[3],
                         const nimbus_cloud* replacement, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!aabb_min || !aabb_max) {
    ctx->err = "update_region: null box";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->obj_stream[scene] = st;
  return nb::update_scene_region(ctx->mem, S, aabb_min, aabb_max, replacement, st);
}

int nimbus_segment(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_segment_params* params,
                   uint32_t* labels, double* edges, uint32_t* edge_labels, int64_t edges_cap,
                   nimbus_segment_counts* counts, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!cloud || !params || !counts || cloud->n < 1 || !cloud->xyz || !cloud->nrm || !labels || edges_cap < 0 ||
      (edges_cap > 0 && (!edges || !edge_labels))) {
    ctx->err = "segment: null argument or empty cloud";
    return NIMBUS_ERR_ARG;
  }
  const nimbus_segment_params& p = *params;
  if (!(p.voxel_size > 0) || p.dv < 1 || p.dv > 4 || p.min_points < 3 || !(p.flat_max >= 0) ||
      !(p.spread_min >= 0) || !(p.join_angle >= 0 && p.join_angle <= 3.1416) || !(p.join_dist >= 0) ||
      !(p.edge_angle >= 0 && p.edge_angle <= 3.1416) || p.edge_min_groups < 1) {
    ctx->err = "segment: parameter out of range";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  nb::StageTimer tm(st);
  const int e0 = tm.mark();
  int rc = NIMBUS_OK;
  {
    // the cloud under a single label: every IE of its voxelisation is one subvoxel's points
    nb::Scratch zs(&ctx->mem, st);
    uint32_t* zero;
    rc = zs.get(&zero, cloud->n);
    if (rc != NIMBUS_OK) return rc;
    if (cudaMemsetAsync(zero, 0, cloud->n * sizeof(uint32_t), st) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "segment: cudaMemsetAsync failed";
      return NIMBUS_ERR_CUDA;
    }
    const nimbus_cloud one{cloud->xyz, cloud->nrm, zero, nullptr, cloud->n};
    nimbus_vox_params vp{};
    const double hs = p.voxel_size / p.dv;
    vp.voxel_size = p.voxel_size;
    vp.dv = p.dv;
    vp.sdf_sigma = 0.5 * hs;
    vp.sdf_eps = 1e-3;
    vp.vis_ignore = hs * std::sqrt(3.0);
    vp.sdf_max_steps = 1;
    auto* S = new nb::SceneObj();
    S->mem = &ctx->mem;
    rc = nb::voxelize_scene(ctx->mem, &one, nullptr, &vp, S, st);
    if (rc == NIMBUS_OK) rc = nb::segment_scene(ctx->mem, S, params, labels, edges, edge_labels, edges_cap, counts, st);
    drop_obj(ctx, S, st);
  }
  const int e1 = tm.mark();
  cudaStreamSynchronize(st);
  counts->ms_total = tm.ms(e0, e1);
  return rc;
}

int nimbus_scene_save(nimbus_ctx* ctx, nimbus_handle scene, const char* path, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  return nb::scene_save(ctx->mem, S, path, (cudaStream_t)stream);
}

int nimbus_scene_load(nimbus_ctx* ctx, const char* path, nimbus_handle* scene_out, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!scene_out) {
    ctx->err = "scene_load: null argument";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  auto* S = new nb::SceneObj();
  S->mem = &ctx->mem;
  int rc = nb::scene_load(ctx->mem, path, S, st);
  if (rc != NIMBUS_OK) {
    drop_obj(ctx, S, st);
    return rc;
  }
  *scene_out = put_obj(ctx, S, st);
  return NIMBUS_OK;
}

int nimbus_trace_coarse(nimbus_ctx* ctx, nimbus_handle scene, const double* tx, int32_t n_tx, const double* rx,
                        int32_t n_rx, const nimbus_trace_params* params, nimbus_handle* coarse_out, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!coarse_out || !params) {
    ctx->err = "trace: null argument";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  auto* C = new nb::CoarseObj();
  C->mem = &ctx->mem;
  C->scene = scene;
  int rc = nb::trace_coarse(ctx->mem, S, tx, n_tx, rx, n_rx, params, C, st, ctx->tune);
  if (rc != NIMBUS_OK && rc != NIMBUS_ERR_OVERFLOW) {
    drop_obj(ctx, C, st);
    return rc;
  }
  *coarse_out = put_obj(ctx, C, st);
  return rc;
}

int nimbus_refine(nimbus_ctx* ctx, nimbus_handle scene, nimbus_handle coarse, const nimbus_refine_params* params,
                  nimbus_handle* paths_out, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!paths_out || !params) {
    ctx->err = "refine: null argument";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  auto* C = get_obj<nb::CoarseObj>(ctx, coarse, nb::OBJ_COARSE);
  if (!C) return NIMBUS_ERR_STATE;
  if (C->scene != scene) {
    ctx->err = "refine: coarse set was traced on another scene";
    return NIMBUS_ERR_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  auto* P = new nb::PathsObj();
  P->mem = &ctx->mem;
  int rc = nb::refine_paths(ctx->mem, S, C, params, P, st, ctx->tune);
  if (rc != NIMBUS_OK) {
    drop_obj(ctx, P, st);
    return rc;
  }
  *paths_out = put_obj(ctx, P, st);
  return NIMBUS_OK;
}

int nimbus_query(nimbus_ctx* ctx, nimbus_handle paths, int32_t which, nimbus_path_counts* counts,
                 const nimbus_path_view* view, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!counts) {
    ctx->err = "query: null counts";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* P = get_obj<nb::PathsObj>(ctx, paths, nb::OBJ_PATHS);
  if (!P) return NIMBUS_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  *counts = P->counts;
  counts->n_paths = P->n_final;
  const int64_t n = which ? P->n_all : P->n_final;
  std::vector<nb::ExactRec> h;
  if (n > 0 && (view || which)) {
    h.resize(n);
    if (which) {
      NB_CUDA(&ctx->err, cudaMemcpyAsync(h.data(), P->all, n * sizeof(nb::ExactRec), cudaMemcpyDeviceToHost, st));
    } else {
      nb::ExactRec* tmp = nullptr;
      int rc = ctx->mem.alloc_n(&tmp, n, st);
      if (rc != NIMBUS_OK) return rc;
      nb::k_gather_exact<<<nb::grid_for(n, 128), 128, 0, st>>>(P->all, P->final_idx, n, tmp);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), tmp, n * sizeof(nb::ExactRec), cudaMemcpyDeviceToHost, st);
      ctx->mem.release(tmp, st);
      if (e != cudaSuccess) return nb::cuda_fail(&ctx->err, e, "query copy");
    }
  }
  NB_CUDA(&ctx->err, cudaStreamSynchronize(st));
  if (which) {
    int64_t nv = 0;
    for (const auto& r : h) nv += r.status == nb::ST_VALID;
    counts->n_refined_valid = nv;
  }
  if (!view) return NIMBUS_OK;
  for (int64_t i = 0; i < n; ++i) {
    const nb::ExactRec& r = h[i];
    if (view->tx) view->tx[i] = (int32_t)r.tx;
    if (view->rx) view->rx[i] = (int32_t)r.rx;
    if (view->n_int) view->n_int[i] = (int32_t)r.n;
    if (view->length) view->length[i] = r.length;
    if (view->delay) view->delay[i] = r.delay;
    if (view->grad) view->grad[i] = r.grad;
    if (view->iters) view->iters[i] = (int32_t)r.iters;
    if (view->status) view->status[i] = (int32_t)r.status;
    for (int q = 0; q < NB_MAXI; ++q) {
      bool in = q < (int)r.n;
      if (view->types) view->types[i * NB_MAXI + q] = in ? (int32_t)((r.types >> q) & 1u) : -1;
      if (view->labels) view->labels[i * NB_MAXI + q] = in ? r.lab[q] : NB_NONE_LABEL;
      if (view->materials) view->materials[i * NB_MAXI + q] = in ? r.mat[q] : 255;
      if (view->ies) view->ies[i * NB_MAXI + q] = in ? (int64_t)r.ie[q] : -1;
      if (view->points)
        for (int a = 0; a < 3; ++a) view->points[(i * NB_MAXI + q) * 3 + a] = in ? r.pts[q][a] : 0.0;
    }
  }
  return NIMBUS_OK;
}

int nimbus_query_coarse(nimbus_ctx* ctx, nimbus_handle coarse, nimbus_path_counts* counts,
                        const nimbus_coarse_view* view, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!counts) {
    ctx->err = "query_coarse: null counts";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* C = get_obj<nb::CoarseObj>(ctx, coarse, nb::OBJ_COARSE);
  if (!C) return NIMBUS_ERR_STATE;
  *counts = C->counts;
  if (!view || C->n == 0) return NIMBUS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = C->n;
  std::vector<uint32_t> tx(n), rx(n), ni(n), ty(n), ie(n * NB_MAXI), lab(n * NB_MAXI);
  std::vector<float> miss(n);
  NB_CUDA(&ctx->err, cudaMemcpyAsync(tx.data(), C->tx, n * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(rx.data(), C->rx, n * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(ni.data(), C->nint, n * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(ty.data(), C->types, n * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(ie.data(), C->ie, n * NB_MAXI * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(lab.data(), C->lab, n * NB_MAXI * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(miss.data(), C->miss, n * 4, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaStreamSynchronize(st));
  for (int64_t i = 0; i < n; ++i) {
    if (view->tx) view->tx[i] = (int32_t)tx[i];
    if (view->rx) view->rx[i] = (int32_t)rx[i];
    if (view->n_int) view->n_int[i] = (int32_t)ni[i];
    if (view->miss) view->miss[i] = miss[i];
    for (int q = 0; q < NB_MAXI; ++q) {
      bool in = q < (int)ni[i];
      if (view->ies) view->ies[i * NB_MAXI + q] = in ? (int64_t)ie[i * NB_MAXI + q] : -1;
      if (view->types) view->types[i * NB_MAXI + q] = in ? (int32_t)((ty[i] >> q) & 1u) : -1;
      if (view->labels) view->labels[i * NB_MAXI + q] = in ? lab[i * NB_MAXI + q] : NB_NONE_LABEL;
    }
  }
  return NIMBUS_OK;
}

int nimbus_scene_info(nimbus_ctx* ctx, nimbus_handle scene, double origin[3], int32_t dims[3], int64_t* n_ie,
                      int64_t* n_points) {
  if (!ctx) return NIMBUS_ERR_ARG;
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  for (int a = 0; a < 3; ++a) {
    if (origin) origin[a] = S->origin[a];
    if (dims) dims[a] = S->dims[a];
  }
  if (n_ie) *n_ie = S->n_ie;
  if (n_points) *n_points = S->n_points;
  return NIMBUS_OK;
}

int nimbus_scene_tables(nimbus_ctx* ctx, nimbus_handle scene, const nimbus_scene_view* view, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!view) {
    ctx->err = "scene_tables: null view";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = S->n_ie;
  const int64_t nc = (int64_t)S->dims[0] * S->dims[1] * S->dims[2];
  std::vector<nb::IERec> ies(n);
  std::vector<uint2> cells(nc);
  std::vector<uint8_t> march(nc);
  if (n) NB_CUDA(&ctx->err, cudaMemcpyAsync(ies.data(), S->d.ies, n * sizeof(nb::IERec), cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(cells.data(), S->d.cells, nc * sizeof(uint2), cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaMemcpyAsync(march.data(), S->d.march, nc, cudaMemcpyDeviceToHost, st));
  NB_CUDA(&ctx->err, cudaStreamSynchronize(st));
  const int dv = S->params.dv;
  const double hs = S->params.voxel_size / dv;
  for (int64_t i = 0; i < n; ++i) {
    const nb::IERec& r = ies[i];
    uint32_t meta, lab, pb, pc;
    std::memcpy(&meta, &r.nrm_meta.w, 4);
    std::memcpy(&lab, &r.rp_lab.w, 4);
    std::memcpy(&pb, &r.bbc_pb.w, 4);
    std::memcpy(&pc, &r.sc_pc.w, 4);
    int kind = (int)(meta & 1u);
    if (view->kind) view->kind[i] = kind;
    if (view->label) view->label[i] = lab;
    if (view->material) view->material[i] = (uint8_t)((meta >> 8) & 0xffu);
    const float sc[3] = {r.sc_pc.x, r.sc_pc.y, r.sc_pc.z};
    int gs[3];
    for (int a = 0; a < 3; ++a) gs[a] = (int)std::floor((sc[a] - S->origin[a]) / hs);
    if (view->gs)
      for (int a = 0; a < 3; ++a) view->gs[3 * i + a] = gs[a];
    if (view->cell)
      view->cell[i] = ((int64_t)(gs[2] / dv) * S->dims[1] + gs[1] / dv) * S->dims[0] + gs[0] / dv;
    if (view->prange) {
      view->prange[2 * i] = kind == 0 ? (int64_t)pb : 0;
      view->prange[2 * i + 1] = kind == 0 ? (int64_t)pc : 0;
    }
    const float rp[3] = {r.rp_lab.x, r.rp_lab.y, r.rp_lab.z}, nn[3] = {r.nrm_meta.x, r.nrm_meta.y, r.nrm_meta.z},
                bb[3] = {r.bbc_pb.x, r.bbc_pb.y, r.bbc_pb.z};
    for (int a = 0; a < 3; ++a) {
      if (view->rp) view->rp[3 * i + a] = rp[a];
      if (view->normal) view->normal[3 * i + a] = nn[a];
      if (view->bbc) view->bbc[3 * i + a] = bb[a];
    }
    if (view->slab) {
      view->slab[4 * i] = r.slab.x;
      view->slab[4 * i + 1] = r.slab.y;
      view->slab[4 * i + 2] = r.slab.z;
      view->slab[4 * i + 3] = r.slab.w;
    }
  }
  for (int64_t c = 0; c < nc; ++c) {
    if (view->cell_begin) view->cell_begin[c] = cells[c].x;
    if (view->cell_count) view->cell_count[c] = (int32_t)cells[c].y;
    if (view->march) view->march[c] = march[c];
  }
  return NIMBUS_OK;
}

int nimbus_release(nimbus_ctx* ctx, nimbus_handle h) {
  if (!ctx) return NIMBUS_ERR_ARG;
  auto it = ctx->objs.find(h);
  if (it == ctx->objs.end()) {
    ctx->err = "release: unknown handle";
    return NIMBUS_ERR_STATE;
  }
  DeviceGuard g(ctx->device);
  drop_obj(ctx, it->second, ctx->obj_stream[h]);
  ctx->objs.erase(it);
  ctx->obj_stream.erase(h);
  return NIMBUS_OK;
}

int nimbus_memory_used(nimbus_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return NIMBUS_ERR_ARG;
  *bytes = ctx->mem.used;
  return NIMBUS_OK;
}

int nimbus_voxelize_static(nimbus_ctx* ctx, const nimbus_cloud* cloud, const nimbus_vox_params* params,
                           const nimbus_static_tables* out, nimbus_static_info* info, void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  DeviceGuard g(ctx->device);
  return nb::voxelize_static(&ctx->err, cloud, params, out, info, (cudaStream_t)stream);
}

static void to_public(const nb::Tuning& t, nimbus_tuning* o) {
  o->level_block = t.level_block;
  o->refine_blocks = t.refine_blocks;
  o->refine_order = t.refine_order;
  o->graph = t.graph;
  o->level_ms = t.level_ms;
  o->refine_ms = t.refine_ms;
  o->level_queue = t.level_queue;
  o->refine_split = t.refine_split;
  o->refine_split_key = t.refine_split_key;
  o->level_help = t.level_help;
  o->level_rx_first = t.level_rx_first;
}

int nimbus_get_tuning(nimbus_ctx* ctx, nimbus_tuning* out) {
  if (!ctx || !out) return NIMBUS_ERR_ARG;
  to_public(ctx->tune, out);
  return NIMBUS_OK;
}

int nimbus_set_tuning(nimbus_ctx* ctx, const nimbus_tuning* t) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!t || !(t->level_block == 128 || t->level_block == 256 || t->level_block == 512) || t->refine_blocks < 0 ||
      t->refine_blocks > 8 ||
      !(t->refine_order >= 0 && t->refine_order <= 2) || !(t->graph == 0 || t->graph == 1) ||
      !(t->level_queue == 0 || t->level_queue == 1) || t->refine_split < 0 || t->refine_split > 65535 ||
      !(t->refine_split_key == 0 || t->refine_split_key == 1) || !(t->level_help == 0 || t->level_help == 1) ||
      !(t->level_rx_first == 0 || t->level_rx_first == 1)) {
    ctx->err = "set_tuning: value out of range";
    return NIMBUS_ERR_ARG;
  }
  ctx->tune.level_block = t->level_block;
  ctx->tune.refine_blocks = t->refine_blocks;
  ctx->tune.refine_order = t->refine_order;
  ctx->tune.graph = t->graph;
  ctx->tune.level_ms = t->level_ms;
  ctx->tune.refine_ms = t->refine_ms;
  ctx->tune.level_queue = t->level_queue;
  ctx->tune.refine_split = t->refine_split;
  ctx->tune.refine_split_key = t->refine_split_key;
  ctx->tune.level_help = t->level_help;
  ctx->tune.level_rx_first = t->level_rx_first;
  return NIMBUS_OK;
}

int nimbus_set_wait_limit(nimbus_ctx* ctx, int64_t cycles) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (cycles < 0) {
    ctx->err = "set_wait_limit: negative limit";
    return NIMBUS_ERR_ARG;
  }
  ctx->tune.wait_limit = (long long)cycles;
  return NIMBUS_OK;
}

int nimbus_autotune(nimbus_ctx* ctx, nimbus_handle scene, const double* tx, int32_t n_tx, const double* rx,
                    int32_t n_rx, const nimbus_trace_params* tp, const nimbus_refine_params* rp, nimbus_tuning* out,
                    void* stream) {
  if (!ctx) return NIMBUS_ERR_ARG;
  if (!tp || !rp) {
    ctx->err = "autotune: null argument";
    return NIMBUS_ERR_ARG;
  }
  DeviceGuard g(ctx->device);
  auto* S = get_obj<nb::SceneObj>(ctx, scene, nb::OBJ_SCENE);
  if (!S) return NIMBUS_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  nb::Tuning best = ctx->tune;
  // level layouts: propagation time of the sample's levels
  double best_lv = -1.0;
  const int blocks[3] = {256, 128, 512};
  for (int lq = 0; lq < 2; ++lq)
  for (int bl : blocks)
  for (int hp = lq == 0 ? 1 : 0; hp >= 0; --hp) {   // the help board exists in the per-depth launch only
    nb::Tuning t = best;
    t.level_block = bl;
    t.level_queue = lq;
    t.level_help = hp;
    auto* C = new nb::CoarseObj();
    C->mem = &ctx->mem;
    C->scene = scene;
    int rc = nb::trace_coarse(ctx->mem, S, tx, n_tx, rx, n_rx, tp, C, st, t);
    const double ms = C->counts.ms_levels;
    drop_obj(ctx, C, st);
    if (rc != NIMBUS_OK) return rc;
    if (best_lv < 0.0 || ms < best_lv) {
      best_lv = ms;
      best.level_block = bl;
      best.level_queue = lq;
      best.level_help = hp;
    }
  }
  {
    // the last level's RX test: tried once, flipped, on the best layout
    nb::Tuning t = best;
    t.level_rx_first = 1 - best.level_rx_first;
    auto* C = new nb::CoarseObj();
    C->mem = &ctx->mem;
    C->scene = scene;
    int rc = nb::trace_coarse(ctx->mem, S, tx, n_tx, rx, n_rx, tp, C, st, t);
    const double ms = C->counts.ms_levels;
    drop_obj(ctx, C, st);
    if (rc != NIMBUS_OK) return rc;
    if (ms < best_lv) {
      best_lv = ms;
      best.level_rx_first = t.level_rx_first;
    }
  }
  best.level_ms = best_lv;
  // refinement layouts, on the coarse set of the chosen level layout
  auto* C = new nb::CoarseObj();
  C->mem = &ctx->mem;
  C->scene = scene;
  int rc = nb::trace_coarse(ctx->mem, S, tx, n_tx, rx, n_rx, tp, C, st, best);
  if (rc != NIMBUS_OK) {
    drop_obj(ctx, C, st);
    return rc;
  }
  double best_rf = -1.0;
  // refinement layouts (all resident blocks per SM: fewer has not won since the flat
  // point list): one launch in each order, then two launches
  struct RefLayout {
    int order, split, key;
  };
  std::vector<RefLayout> layouts = {{0, 0, 0}, {1, 0, 0}, {2, 0, 0}};
  for (int sl : {64, 128, 512})
    for (int od : {0, 1})
      for (int key : {0, 1}) layouts.push_back({od, sl, key});
  for (const RefLayout& L : layouts) {
    if (rc != NIMBUS_OK) break;   // an error ends the search (reported below)
    nb::Tuning t = best;
    t.refine_blocks = 0;
    t.refine_order = L.order;
    t.refine_split = L.split;
    t.refine_split_key = L.key;
    auto* P = new nb::PathsObj();
    P->mem = &ctx->mem;
    rc = nb::refine_paths(ctx->mem, S, C, rp, P, st, t);
    const double ms = P->counts.ms_refine;
    drop_obj(ctx, P, st);
    if (rc != NIMBUS_OK) continue;
    if (best_rf < 0.0 || ms < best_rf) {
      best_rf = ms;
      best.refine_blocks = 0;
      best.refine_order = L.order;
      best.refine_split = L.split;
      best.refine_split_key = L.key;
    }
  }
  drop_obj(ctx, C, st);
  if (rc != NIMBUS_OK) return rc;
  best.refine_ms = best_rf;
  ctx->tune = best;
  if (out) to_public(best, out);
  return NIMBUS_OK;
}

int nimbus_kernel_launches(int64_t* count) {
  if (!count) return NIMBUS_ERR_ARG;
  *count = (int64_t)nb::g_launches.load();
  return NIMBUS_OK;
}

int nimbus_device_allocations(int64_t* count) {
  if (!count) return NIMBUS_ERR_ARG;
  *count = (int64_t)nb::g_allocs.load();
  return NIMBUS_OK;
}

}  // extern "C"
