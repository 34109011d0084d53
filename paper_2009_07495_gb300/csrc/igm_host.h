// igm_host.h -- host-side objects shared by the C-ABI translation units
// (internal): the device-memory arena, the handle of one system and the
// batch (tile tables plus captured launch graphs) of one or more systems.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "igm_launch.h"

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      cudaGetLastError();                                                         \
      return fail(IGM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
    }                                                                             \
  } while (0)

#define CKL()                                                                     \
  do {                                                                            \
    cudaError_t e_ = igm::take_launch_error();                                    \
    cudaError_t l_ = cudaGetLastError();                                          \
    if (e_ == cudaSuccess) e_ = l_;                                               \
    if (e_ != cudaSuccess) return fail(IGM_ECUDA, "launch: %s", cudaGetErrorString(e_)); \
  } while (0)

// NVTX ranges around the host-side phases (build variant "nvtx", -DIGM_NVTX;
// nothing otherwise): visible in a profiler's timeline
#ifdef IGM_NVTX
#include <nvtx3/nvToolsExt.h>
namespace igm {
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace igm
#define IGM_RANGE_CAT2(a, b) a##b
#define IGM_RANGE_CAT(a, b) IGM_RANGE_CAT2(a, b)
#define IGM_RANGE(name) ::igm::NvtxRange IGM_RANGE_CAT(igm_range_, __LINE__)(name)
#else
#define IGM_RANGE(name) ((void)0)
#endif

using igm::BatchDev;
using igm::SysDev;
using igm::SysScal;

// A bump allocator over one cudaMalloc: 256-byte aligned sub-buffers.
struct Arena {
  char *base = nullptr;
  size_t size = 0, off = 0;
  std::vector<std::pair<void **, size_t>> plan;
  template <class T>
  void want(T **p, size_t count) { plan.push_back({(void **)p, count * sizeof(T)}); }
  size_t total() const {
    size_t t = 0;
    for (auto &q : plan) t += (q.second + 255) & ~size_t(255);
    return t + 256;
  }
  cudaError_t commit() {
    size = total();
    cudaError_t e = cudaMalloc((void **)&base, size);
    if (e != cudaSuccess) return e;
    size_t o = 0;
    for (auto &q : plan) {
      *q.first = base + o;
      o += (q.second + 255) & ~size_t(255);
    }
    plan.clear();
    return cudaSuccess;
  }
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
  }
};

struct Batch;

struct igm_handle_s {
  int n = 0, nnz = 0;
  igm_params prm{};
  Arena arena, arena2;   // system data; substitution schedules
  Arena arena3;          // the substitutions' packed group blocks
  SysDev hs{};           // host copy of the descriptor (device pointers)
  SysDev *d_sys = nullptr;
  SysScal *d_sc = nullptr;
  unsigned *d_err = nullptr;
  Batch *solo = nullptr;  // batch of one, with its captured graphs
  int *perm = nullptr;    // multicolour order: perm[new] = old (device)
  double *ptmp = nullptr; // staging vector of the permutation (device)
  int ran_fuse = 0, ran_snap = 0;  // launch configuration of the last solve
};

// right-hand sides in, solutions out, in the caller's row order
igm_status load_vec(igm_handle h, double *dst, const double *src, cudaStream_t s);
igm_status store_vec(igm_handle h, double *dst, const double *src, cudaStream_t s);

struct Batch {
  std::vector<igm_handle> hs;
  long long nodes_check = 0, nodes_cycle = 0;
  int m = 0, any_ilu = 0, inner = 0, max_chunk = 0;
  int fuse_ok = 0;        // the fused Arnoldi kernel applies
  int snap = 0;           // the Arnoldi plan's snap (mgs_plan)
  bool tune = false;      // the autotuner still has to choose
  Arena arena;
  Arena plan_arena;       // the Arnoldi step's plan (set_plan)
  BatchDev bd{};
  int *h_nact = nullptr;  // pinned
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_check = nullptr, g_cycle = nullptr;
  ~Batch() {
    if (g_check) cudaGraphExecDestroy(g_check);
    if (g_cycle) cudaGraphExecDestroy(g_cycle);
    if (cap) cudaStreamDestroy(cap);
    if (h_nact) cudaFreeHost(h_nact);
    arena.release();
    plan_arena.release();
  }
};


// shared helpers (igm_api.cu)
extern thread_local std::string g_err;
igm_status build_batch(const std::vector<igm_handle> &hs, Batch **out);
igm_status set_plan(Batch *b, int snap);
igm_status fail(igm_status st, const char *fmt, ...);
extern std::atomic<long long> g_launches;
void enqueue_inner_host(Batch *b, cudaStream_t st);
igm_status ir_init_host(Batch *b, cudaStream_t st);
igm_status ir_finish_host(Batch *b, cudaStream_t st);
igm_status collect_host(igm_handle h, igm_report *rep, cudaStream_t st);
long long handle_bytes_estimate(int n, int nnz, const igm_params *p);
