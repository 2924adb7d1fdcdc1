// Host-side internals of the CUDA library: device-memory accounting, the sort and
// scan primitives and the launch wrappers of each stage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <unordered_map>
#include <vector>

#include "nimbus_internal.cuh"

namespace nb {

// Device memory of one context, stream-ordered (cudaMallocAsync), bounded by a budget.
struct Mem {
  size_t budget = 0, used = 0, peak = 0;
  std::unordered_map<void*, size_t> sizes;
  std::string* err = nullptr;
  struct GraphCache* graphs = nullptr;   // the context's CUDA graphs (may be null)
  int alloc(void** p, size_t bytes, cudaStream_t st);
  void release(void* p, cudaStream_t st);
  template <class T>
  int alloc_n(T** p, size_t n, cudaStream_t st) {
    return alloc(reinterpret_cast<void**>(p), n * sizeof(T) + 16, st);
  }
};

// A list of device allocations released together.  With an arena set, buffers are
// carved from that preallocated device region instead (nothing is allocated).
struct Scratch {
  Mem* mem;
  cudaStream_t st;
  std::vector<void*> ptrs;
  char* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  Scratch(Mem* m, cudaStream_t s) : mem(m), st(s) {}
  ~Scratch() {
    for (void* p : ptrs) mem->release(p, st);
  }
  // bytes an arena gives one get of n elements of size elem
  static size_t arena_block(size_t n, size_t elem) { return (n * elem + 16 + 255) & ~(size_t)255; }
  template <class T>
  int get(T** p, size_t n) {
    if (arena) {
      size_t bytes = arena_block(n, sizeof(T));
      if (arena_used + bytes > arena_cap) {
        if (mem && mem->err) *mem->err = "static scratch exhausted";
        return NIMBUS_ERR_ARG;
      }
      *p = reinterpret_cast<T*>(arena + arena_used);
      arena_used += bytes;
      return NIMBUS_OK;
    }
    int rc = mem->alloc_n(p, n, st);
    if (rc == NIMBUS_OK) ptrs.push_back(*p);
    return rc;
  }
};

int cuda_fail(std::string* err, cudaError_t e, const char* what);
#define NB_CUDA(err, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::nb::cuda_fail(err, e_, #call); \
  } while (0)
// Kernel launches made by the library (process-wide), for launch accounting.
extern std::atomic<long long> g_launches;
// Device allocations made by the library (process-wide), for allocation accounting.
extern std::atomic<long long> g_allocs;
#define NB_LAUNCHED(err)                 \
  do {                                   \
    ::nb::g_launches.fetch_add(1);       \
    NB_CUDA(err, cudaGetLastError());    \
  } while (0)
#define NB_TRY(call)               \
  do {                             \
    int rc_ = (call);              \
    if (rc_ != NIMBUS_OK) return rc_; \
  } while (0)

int num_sms();

// CUDA events recorded on one stream to time stages of kernels (read after a sync).
struct StageTimer {
  cudaEvent_t ev[16];
  bool owned[16];
  int n = 0;
  cudaStream_t st;
  explicit StageTimer(cudaStream_t s) : st(s) {}
  ~StageTimer() {
    for (int i = 0; i < n; ++i)
      if (owned[i]) cudaEventDestroy(ev[i]);
  }
  int mark() {
    if (n >= 16) return n - 1;
    cudaEventCreate(&ev[n]);
    owned[n] = true;
    cudaEventRecord(ev[n], st);
    return n++;
  }
  // An event to record later with record(); created here because a stream capture
  // may not create events.
  int make() {
    if (n >= 16) return n - 1;
    cudaEventCreate(&ev[n]);
    owned[n] = true;
    return n++;
  }
  // An event owned elsewhere (it outlives the timer), to record later with record().
  int adopt(cudaEvent_t e) {
    if (n >= 16) return n - 1;
    ev[n] = e;
    owned[n] = false;
    return n++;
  }
  // Record event i on q.  On a capturing stream the record becomes a node of the
  // graph (an external record), so the event is stamped when the graph runs.
  void record(int i, cudaStream_t q) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(q, &cs);
    cudaEventRecordWithFlags(ev[i], q,
                             cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  double ms(int a, int b) {
    float m = 0.f;
    if (a < 0 || b < 0 || a >= n || b >= n || cudaEventElapsedTime(&m, ev[a], ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return 0.0;
    }
    return (double)m;
  }
};

// Exclusive prefix sum of n 32-bit counts; total (device, may be null) receives the sum.
int exclusive_scan(Scratch& sc, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total);

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.  The
// sorted pairs end in (keys, vals); keys_alt / vals_alt are work buffers of n.
int radix_sort(Scratch& sc, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
               int64_t n, int bits);

// Arena bytes that exclusive_scan (with or without a total) and radix_sort take from a
// Scratch in arena mode for n items.
size_t scan_arena_bytes(int64_t n, bool total);
size_t radix_arena_bytes(int64_t n, int bits);

// The CUDA graphs of one context: a private capture stream and one executable graph
// per stretch site.  A new capture of a site refreshes its executable in place
// (cudaGraphExecUpdate) when the shape is unchanged -- only pointers, sizes and
// launch parameters differ -- and is instantiated afresh otherwise.  Every stretch
// is followed by a host sync before its site is captured again, so no executable is
// updated while it runs.
enum { GRAPH_TRACE = 0, GRAPH_REFINE = 1, GRAPH_DEDUP = 2, N_GRAPH_SITES = 3 };
// The stage events a site records live here too: a kept executable refers to them.
enum { GRAPH_EVENTS = 6 };
struct GraphCache {
  cudaStream_t cs = nullptr;
  cudaGraphExec_t exec[N_GRAPH_SITES] = {};
  cudaEvent_t ev[N_GRAPH_SITES][GRAPH_EVENTS] = {};
  long long instantiated = 0, updated = 0;
  cudaEvent_t event(int site, int k) {
    if (!ev[site][k]) cudaEventCreate(&ev[site][k]);
    return ev[site][k];
  }
  void release() {
    for (cudaGraphExec_t& e : exec)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
    for (auto& row : ev)
      for (cudaEvent_t& e : row)
        if (e) {
          cudaEventDestroy(e);
          e = nullptr;
        }
    if (cs) cudaStreamDestroy(cs);
    cs = nullptr;
  }
  ~GraphCache() { release(); }
};

// Stage event k of a stretch site for tm: the context's own when it keeps graphs,
// else one that tm creates and destroys.
inline int stretch_event(StageTimer& tm, Mem& mem, int site, int k) {
  return mem.graphs ? tm.adopt(mem.graphs->event(site, k)) : tm.make();
}

// A stretch of stream work with no host round trip: fn(q) issues it on stream q.
// With graph = false it goes straight onto st.  With graph = true it is captured on a
// private stream into one CUDA graph and launched on st, so the whole stretch is one
// graph launch; with the context's cache (mem.graphs) the executable of `site` is
// kept between calls.  fn must not allocate, synchronise or copy to or from pageable
// host memory; its Scratch buffers come from an arena.
template <class F>
int run_stretch(Mem& mem, cudaStream_t st, bool graph, int site, F&& fn) {
  std::string* err = mem.err;
  if (!graph) return fn(st);
  GraphCache* gc = mem.graphs;
  cudaStream_t cs = gc ? gc->cs : nullptr;
  if (!cs) {
    NB_CUDA(err, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (gc) gc->cs = cs;
  }
  struct StreamDel {
    cudaStream_t s;
    ~StreamDel() {
      if (s) cudaStreamDestroy(s);
    }
  } del{gc ? nullptr : cs};
  NB_CUDA(err, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const int rc = fn(cs);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &g);
  if (rc != NIMBUS_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  }
  NB_CUDA(err, ec);
  cudaGraphExec_t local = nullptr;
  cudaGraphExec_t& ge = gc ? gc->exec[site] : local;
  if (ge) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ge, g, &info) == cudaSuccess) {
      ++gc->updated;
    } else {
      cudaGetLastError();
      cudaGraphExecDestroy(ge);
      ge = nullptr;
    }
  }
  if (!ge) {
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0ull);
    if (ei != cudaSuccess) {
      ge = nullptr;
      cudaGraphDestroy(g);
      return cuda_fail(err, ei, "cudaGraphInstantiate");
    }
    if (gc) ++gc->instantiated;
  }
  cudaGraphDestroy(g);
  const cudaError_t el = cudaGraphLaunch(ge, st);
  if (!gc) cudaGraphExecDestroy(ge);   // freed once the launch completes
  NB_CUDA(err, el);
  return NIMBUS_OK;
}

// ----------------------------------------------------------------------------- objects
enum { OBJ_SCENE = 1, OBJ_COARSE = 2, OBJ_PATHS = 3 };

struct Obj {
  int kind;
  Mem* mem = nullptr;
  std::vector<void*> bufs;   // device buffers owned by the object
  explicit Obj(int k) : kind(k) {}
  virtual ~Obj() {}
  template <class T>
  int own(T** p, size_t n, cudaStream_t st) {
    int rc = mem->alloc_n(p, n, st);
    if (rc == NIMBUS_OK) bufs.push_back(*p);
    return rc;
  }
  void free_all(cudaStream_t st) {
    for (void* p : bufs) mem->release(p, st);
    bufs.clear();
  }
};

// A voxelised scene (Section 2.1): grid, entity table, grouped points, voxel ranges,
// march field, plus the input cloud kept on the device for region updates.
struct SceneObj : Obj {
  SceneObj() : Obj(OBJ_SCENE) {}
  DScene d{};
  nimbus_vox_params params{};
  double origin[3] = {0, 0, 0};
  int dims[3] = {0, 0, 0};
  int64_t n_ie = 0, n_slots = 0, n_points = 0;
  // device copies of the input
  float* xyz = nullptr;
  float* nrm = nullptr;
  uint32_t* label = nullptr;
  uint8_t* material = nullptr;
  std::vector<double> edges_h;
  std::vector<uint32_t> edge_label_h;
  uint32_t max_label = 0;
  // derived tables (owned; freed and rebuilt by region updates)
  std::vector<void*> table_bufs;
  uint32_t* ie_start = nullptr;   // [n_ie + 1] first entry of each IE in the grouped point table
  uint32_t* ie_cell = nullptr;    // [n_ie] voxel of each IE
};

// Coarse paths after the kappa limit (Section 2.2.3), structure of arrays.
struct CoarseObj : Obj {
  CoarseObj() : Obj(OBJ_COARSE) {}
  nimbus_handle scene = 0;
  int n_tx = 0, n_rx = 0;
  double* txd = nullptr;     // [n_tx*3] device
  double* rxd = nullptr;     // [n_rx*3] device
  int64_t n = 0;
  uint32_t* tx = nullptr;
  uint32_t* rx = nullptr;
  uint32_t* nint = nullptr;
  uint32_t* types = nullptr; // bit k set: interaction k is a diffraction
  uint32_t* ie = nullptr;    // [n*NB_MAXI]
  uint32_t* lab = nullptr;   // [n*NB_MAXI]
  float* miss = nullptr;
  uint32_t* gid = nullptr;   // group of (tx, rx, types, labels)
  uint32_t n_groups_cap = 0;
  int max_refl = NB_MAXI;    // reflection limit of the trace (bounds the reflections of every path)
  nimbus_path_counts counts{};
};

// One refined path (Section 2.3).
struct ExactRec {
  double pts[NB_MAXI][3];
  double length, delay, grad;
  uint32_t tx, rx, n, types, status, iters, gid, pad;
  uint32_t lab[NB_MAXI];
  uint32_t ie[NB_MAXI];
  uint8_t mat[NB_MAXI];
};

struct PathsObj : Obj {
  PathsObj() : Obj(OBJ_PATHS) {}
  int64_t n_all = 0, n_final = 0;
  ExactRec* all = nullptr;       // one per refined coarse path
  uint32_t* final_idx = nullptr; // indices into all, final order
  nimbus_path_counts counts{};
};

// Launch layout of the propagation levels and the refinement (result-neutral).
struct Tuning {
  int level_block = 512;
  int refine_blocks = 0;   // 0: as many as fit
  int refine_order = 1;
  int graph = 1;           // issue each host-free stretch of a call as one CUDA graph
  int level_queue = 0;     // 1: all propagation depths in one launch (a task queue across levels)
  int refine_split = 0;    // > 0: two-phase refinement, phase 1 capped at this many iterations
  int refine_split_key = 0;  // phase 2 order: 0 cost per iteration, 1 predicted remaining time
  int level_help = 1;      // per-depth levels: idle warps of a block walk its running cones' visibility rays
  int level_rx_first = 1;   // last level: skip cones none of whose reachable RXs sees the apex
  long long wait_limit = 0;  // cycles after which a level wait gives up (0: the defaults); for tests
  double level_ms = 0, refine_ms = 0;
};

int trace_coarse(Mem& mem, SceneObj* S, const double* tx, int n_tx, const double* rx, int n_rx,
                 const nimbus_trace_params* p, CoarseObj* out, cudaStream_t st, const Tuning& tn);
int refine_paths(Mem& mem, SceneObj* S, CoarseObj* C, const nimbus_refine_params* p, PathsObj* out,
                 cudaStream_t st, const Tuning& tn);

int voxelize_scene(Mem& mem, const nimbus_cloud* cloud, const nimbus_edges* edges, const nimbus_vox_params* p,
                   SceneObj* out, cudaStream_t st);
int scene_save(Mem& mem, SceneObj* S, const char* path, cudaStream_t st);
// Automatic labels and exterior edges (nimbus_segment) of a scene voxelised under a
// single label: each of its IEs is the point group of one subvoxel.
int segment_scene(Mem& mem, SceneObj* S, const nimbus_segment_params* p, uint32_t* labels_out, double* edges_out,
                  uint32_t* edge_labels_out, int64_t edges_cap, nimbus_segment_counts* counts, cudaStream_t st);
int scene_load(Mem& mem, const char* path, SceneObj* S, cudaStream_t st);
int update_scene_region(Mem& mem, SceneObj* s, const double lo[3], const double hi[3],
                        const nimbus_cloud* repl, cudaStream_t st);

// Voxelisation into caller buffers with every intermediate in a fixed device array.
int voxelize_static(std::string* err, const nimbus_cloud* cloud, const nimbus_vox_params* p,
                    const nimbus_static_tables* out, nimbus_static_info* info, cudaStream_t st);

bool is_device_ptr(const void* p);
// Copy n bytes of a host or device input into a device buffer.
int copy_in(std::string* err, void* dst, const void* src, size_t n, cudaStream_t st);

inline int bits_for(uint64_t max_value) {
  int b = 0;
  while (b < 64 && (max_value >> b) != 0) ++b;
  return b;
}

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace nb
