// api.cu -- the extern "C" boundary of liblens.so (declared in include/lens.h)
// plus the host plumbing: status codes, thread-local error text, device
// allocation through the caller's allocator, host-side fault injection
// (LENS_FAULT=alloc@K | launch@K), and the chunk driver of lens_ipm_map
// (Sec. 2.4: split the image plane into chunks, deflect each chunk with the
// FMM, apportion its cells with IPM, accumulate one map).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lens_internal.h"
#include "images.h"
#include "potential.h"

namespace lens {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_alloc_count{0}, g_launch_count{0};

struct FaultSpec {
  long long alloc_at = -1, launch_at = -1;
  FaultSpec() {
    const char* e = std::getenv("LENS_FAULT");
    if (!e) return;
    long long k = 0;
    if (std::sscanf(e, "alloc@%lld", &k) == 1) alloc_at = k;
    else if (std::sscanf(e, "launch@%lld", &k) == 1) launch_at = k;
  }
};
const FaultSpec& fault_spec() {
  static FaultSpec f;
  return f;
}
}  // namespace

void fail(lens_status st, const std::string& msg) { throw Error{st, msg}; }
void set_last_error(const std::string& msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      fail(LENS_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    fail(LENS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void after_launch(const char* name) {
  const long long k = ++g_launch_count;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(LENS_ECUDA, std::string("launch ") + name + ": " + cudaGetErrorString(e));
  if (fault_spec().launch_at == k) fail(LENS_EFAULT_INJECTED, std::string("injected launch fault at ") + name);
}

long long launch_count() { return g_launch_count.load(); }

void fault_point_alloc() {
  const long long k = ++g_alloc_count;
  if (fault_spec().alloc_at == k) fail(LENS_EFAULT_INJECTED, "injected allocation fault");
}

// Without a caller allocator, device memory comes from one stream-ordered
// pool per device owned by the library.  Freed blocks stay reserved for reuse
// (up to kPoolKeepBytes across synchronisations), so the next plan or map
// reuses them instead of mapping fresh memory: with the default pool, which
// returns freed memory at every synchronisation, the tree build's allocations
// between its size read-backs cost ~0.7 ms per build.
constexpr uint64_t kPoolKeepBytes = 16ull << 30;

static cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  LENS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  LENS_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = kPoolKeepBytes;
  LENS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

void* DeviceAlloc::alloc(size_t bytes) {
  fault_point_alloc();
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (custom) {
    p = a.alloc(bytes, (void*)stream, a.ctx);
    if (!p) fail(LENS_ENOMEM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(LENS_ENOMEM, "cudaMallocFromPoolAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  return p;
}

void DeviceAlloc::release(void* p) {
  if (!p) return;
  if (custom) a.free(p, (void*)stream, a.ctx);
  else cudaFreeAsync(p, stream);
}

}  // namespace lens

using namespace lens;

struct lens_plan {
  Plan P;
};

#define LENS_API_BEGIN try {
#define LENS_API_END                                   \
  }                                                    \
  catch (const Error& e) {                             \
    set_last_error(e.msg);                             \
    return e.status;                                   \
  }                                                    \
  catch (const std::exception& e) {                    \
    set_last_error(std::string("internal: ") + e.what()); \
    return LENS_ECUDA;                                 \
  }                                                    \
  set_last_error("");                                  \
  return LENS_OK;

namespace {
// lens_ipm_map with a float32-bulk plan and no flag: the fused path or not
constexpr bool kFusedDefault = false;

void need(bool ok, const char* msg) {
  if (!ok) fail(LENS_EINVAL, msg);
}
cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void check_grid(const Plan& P, const lens_grid* g) {
  need(g != nullptr, "grid is NULL");
  need(std::isfinite(g->x0) && std::isfinite(g->y0) && std::isfinite(g->h) && g->h > 0,
       "grid x0, y0 must be finite and h > 0");
  need(g->nx >= 1 && g->ny >= 1, "grid needs nx >= 1 and ny >= 1");
  const double x1 = g->x0 + (double)g->nx * g->h, y1 = g->y0 + (double)g->ny * g->h;
  double lo0, hi0, lo1, hi1;
  if (P.has_target) {
    lo0 = P.target[0]; hi0 = P.target[1]; lo1 = P.target[2]; hi1 = P.target[3];
    if (!(g->x0 >= lo0 && x1 <= hi0 && g->y0 >= lo1 && y1 <= hi1))
      fail(LENS_EDOMAIN, "grid extends beyond the plan's target box");
  } else {
    lo0 = P.root_lo[0]; hi0 = P.root_lo[0] + P.root_size;
    lo1 = P.root_lo[1]; hi1 = P.root_lo[1] + P.root_size;
    if (!(g->x0 >= lo0 && x1 < hi0 && g->y0 >= lo1 && y1 < hi1))
      fail(LENS_EDOMAIN, "grid extends beyond the plan's root box");
  }
}
}  // namespace

void lens::wait_expansions(Plan& P, cudaStream_t s) {
  if (P.ev_fmm) LENS_CUDA(cudaStreamWaitEvent(s, P.ev_fmm, 0));
}
void lens::wait_tree(Plan& P, cudaStream_t s) {
  if (P.ev_tree) LENS_CUDA(cudaStreamWaitEvent(s, P.ev_tree, 0));
}

extern "C" {

const char* lens_last_error(void) { return g_last_error.c_str(); }

const char* lens_version(void) { return "lens-fmm-gb300 0.1 (sm_103a)"; }

lens_status lens_fmm_build(const double* stars_xy, const double* masses, int64_t n,
                           double kappa_s, double gamma, const lens_build_opts* opts,
                           const lens_allocator* allocator, void* stream, lens_plan** out) {
  lens_plan* plan = nullptr;
  LENS_API_BEGIN
  need(out != nullptr, "out is NULL");
  *out = nullptr;
  need(opts != nullptr, "opts is NULL");
  need(stars_xy != nullptr && masses != nullptr, "stars or masses is NULL");
  need(n >= 1, "need at least one star");
  need(n < (int64_t)INT32_MAX, "too many stars");
  need(opts->p >= 1 && opts->p <= kMaxOrder, "p must be in 1..64");
  need(opts->leaf_size >= 1 && opts->leaf_size <= 1024, "leaf_size must be in 1..1024");
  need(opts->prec == LENS_FP64 || opts->prec == LENS_FP32_BULK, "prec must be LENS_FP64 or LENS_FP32_BULK");
  need(opts->max_depth >= 0 && opts->max_depth <= kMaxDepth, "max_depth must be in 0..28");
  need(std::isfinite(kappa_s) && std::isfinite(gamma), "kappa_s, gamma must be finite");
  if (opts->has_target_box) {
    const double* t = opts->target_box;
    need(std::isfinite(t[0]) && std::isfinite(t[1]) && std::isfinite(t[2]) && std::isfinite(t[3]) &&
             t[0] <= t[1] && t[2] <= t[3],
         "target_box must be finite with min <= max");
  }
  plan = new lens_plan();
  Plan& P = plan->P;
  cudaGetDevice(&P.device);
  P.da.stream = S(stream);
  if (allocator && allocator->alloc && allocator->free) {
    P.da.a = *allocator;
    P.da.custom = true;
  }
  P.n = n;
  P.p = opts->p;
  P.leaf = opts->leaf_size;
  P.prec = opts->prec;
  P.depth = opts->max_depth ? opts->max_depth : kMaxDepth;
  P.kappa_s = kappa_s;
  P.gamma = gamma;
  P.has_target = opts->has_target_box != 0;
  if (P.has_target) std::memcpy(P.target, opts->target_box, sizeof(P.target));
  LENS_CUDA(cudaEventCreate(&P.ev_start));
  LENS_CUDA(cudaEventCreate(&P.ev_tree));
  LENS_CUDA(cudaEventCreateWithFlags(&P.ev_boxes, cudaEventDisableTiming));
  LENS_CUDA(cudaEventCreateWithFlags(&P.ev_up, cudaEventDisableTiming));
  LENS_CUDA(cudaEventCreate(&P.ev_lists));
  LENS_CUDA(cudaEventCreate(&P.ev_fmm));
  LENS_CUDA(cudaEventCreate(&P.ev_far0));
  LENS_CUDA(cudaEventCreate(&P.ev_far1));
  LENS_CUDA(cudaEventRecord(P.ev_start, S(stream)));
  const long long l0 = launch_count();
  // The boxes on the caller's stream.  The upward pass (P2M, M2M) needs only
  // the boxes: it runs on the plan's low-priority stream, and the
  // interaction lists on its high-priority stream, so that the lists (short
  // launches and two read-backs) are not queued behind the float64 upward
  // blocks.  The far field then waits for both, the float32 near-field
  // staging for the lists only (on the caller's stream, beside the far field).
  tree_build_boxes(P, stars_xy, masses, S(stream));  // and the translation tables
  fmm_alloc(P);
  LENS_CUDA(cudaEventRecord(P.ev_boxes, S(stream)));
  int lo_prio = 0, hi_prio = 0;
  LENS_CUDA(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
  LENS_CUDA(cudaStreamCreateWithPriority(&P.up_stream, cudaStreamNonBlocking, lo_prio));
  LENS_CUDA(cudaStreamCreateWithPriority(&P.fmm_stream, cudaStreamNonBlocking, hi_prio));
  LENS_CUDA(cudaStreamWaitEvent(P.up_stream, P.ev_boxes, 0));
  LENS_CUDA(cudaStreamWaitEvent(P.fmm_stream, P.ev_boxes, 0));
  fmm_p2m(P, P.up_stream);
  fmm_m2m(P, P.up_stream);
  LENS_CUDA(cudaEventRecord(P.ev_up, P.up_stream));
  {
    // the lists' allocations are ordered on the stream that uses them
    struct Restore {
      DeviceAlloc& da;
      cudaStream_t s;
      ~Restore() { da.stream = s; }
    } restore{P.da, P.da.stream};
    P.da.stream = P.fmm_stream;
    tree_build_lists(P, P.fmm_stream);
  }
  LENS_CUDA(cudaEventRecord(P.ev_lists, P.fmm_stream));
  LENS_CUDA(cudaStreamWaitEvent(P.fmm_stream, P.ev_up, 0));
  fmm_downward(P, P.fmm_stream);
  LENS_CUDA(cudaStreamWaitEvent(S(stream), P.ev_lists, 0));
  if (P.prec == LENS_FP32_BULK) {
    eval32_alloc(P);
    eval32_prepare_tree(P, S(stream));
  }
  LENS_CUDA(cudaEventRecord(P.ev_tree, S(stream)));
  LENS_CUDA(cudaStreamWaitEvent(P.fmm_stream, P.ev_tree, 0));
  if (P.prec == LENS_FP32_BULK) eval32_prepare_expansions(P, P.fmm_stream);
  LENS_CUDA(cudaEventRecord(P.ev_fmm, P.fmm_stream));
  P.build_launches = launch_count() - l0;
  *out = plan;
  plan = nullptr;
  }
  catch (const Error& e) {
    set_last_error(e.msg);
    if (plan) lens_plan_destroy(plan);
    return e.status;
  }
  catch (const std::exception& e) {
    set_last_error(std::string("internal: ") + e.what());
    if (plan) lens_plan_destroy(plan);
    return LENS_ECUDA;
  }
  set_last_error("");
  return LENS_OK;
}

void lens_plan_destroy(lens_plan* plan) {
  if (!plan) return;
  Plan& P = plan->P;
  // the plan's arrays may be in use on any stream the caller evaluated on
  cudaDeviceSynchronize();
  for (void* p : P.owned) P.da.release(p);
  cudaStreamSynchronize(P.da.stream);
  P.ev_clear();
  if (P.fmm_stream) cudaStreamDestroy(P.fmm_stream);
  if (P.up_stream) cudaStreamDestroy(P.up_stream);
  for (cudaEvent_t e : {P.ev_start, P.ev_boxes, P.ev_tree, P.ev_fmm, P.ev_far0, P.ev_far1,
                        P.ev_up, P.ev_lists})
    if (e) cudaEventDestroy(e);
  delete plan;
}

lens_status lens_plan_info_get(const lens_plan* plan, lens_plan_info* info) {
  LENS_API_BEGIN
  need(plan && info, "NULL argument");
  const Plan& P = plan->P;
  std::memset(info, 0, sizeof(*info));
  info->n_stars = P.n;
  info->n_boxes = P.nb;
  info->n_active_boxes = P.n_active;
  info->n_active_leaves = P.n_active_leaves;
  info->n_v = P.nV; info->n_x = P.nX; info->n_u = P.nU; info->n_w = P.nW;
  info->u_stars = P.u_stars;
  info->levels = P.nlevels;
  info->p = P.p; info->leaf_size = P.leaf; info->prec = P.prec;
  info->root_lo[0] = P.root_lo[0]; info->root_lo[1] = P.root_lo[1];
  info->root_size = P.root_size;
  info->device_bytes = P.device_bytes;
  // the expansions may still be running on the plan's stream
  float ms = 0.f, ms_tree = 0.f;
  if (P.ev_fmm) {
    LENS_CUDA(cudaEventSynchronize(P.ev_fmm));
    LENS_CUDA(cudaEventElapsedTime(&ms, P.ev_start, P.ev_fmm));
    LENS_CUDA(cudaEventElapsedTime(&ms_tree, P.ev_start, P.ev_lists));
  }
  info->ms_build = ms;
  info->ms_tree = ms_tree;
  info->ms_far_local = 0.0;
  if (P.ev_fmm && P.n_active > 0) {
    float mf = 0.f;
    LENS_CUDA(cudaEventElapsedTime(&mf, P.ev_far0, P.ev_far1));
    info->ms_far_local = mf;
  }
  info->build_launches = P.build_launches;
  info->n_leaves = -1;  // not tracked separately (n_active_leaves is)
  LENS_API_END
}

lens_status lens_deflect(lens_plan* plan, const double* rays_xy, int64_t m, double* y_out,
                         double* jac_out, void* stream) {
  LENS_API_BEGIN
  need(plan != nullptr, "plan is NULL");
  need(m >= 0, "m must be >= 0");
  if (m == 0) return LENS_OK;
  need(rays_xy && y_out, "rays or y_out is NULL");
  need(m < (int64_t)INT32_MAX, "too many rays in one call");
  Plan& P = plan->P;
  P.da.stream = S(stream);
  evaluate_rays(P, rays_xy, m, y_out, jac_out, S(stream));
  LENS_API_END
}

lens_status lens_potential(lens_plan* plan, const double* rays_xy, int64_t m, double* psi_out,
                           void* stream) {
  LENS_API_BEGIN
  need(plan != nullptr, "plan is NULL");
  need(m >= 0, "m must be >= 0");
  if (m == 0) return LENS_OK;
  need(rays_xy && psi_out, "rays or psi_out is NULL");
  Plan& P = plan->P;
  P.da.stream = S(stream);
  evaluate_potential(P, rays_xy, m, psi_out, S(stream));
  LENS_API_END
}

lens_status lens_deflect_grid(lens_plan* plan, const lens_grid* grid, int64_t row0, int64_t nrows,
                              double* y_out, double* jac_out, void* stream) {
  LENS_API_BEGIN
  need(plan != nullptr, "plan is NULL");
  Plan& P = plan->P;
  check_grid(P, grid);
  need(row0 >= 0 && nrows >= 0 && row0 + nrows <= grid->ny + 1, "row range outside the grid");
  if (nrows == 0) return LENS_OK;
  need(y_out != nullptr, "y_out is NULL");
  P.da.stream = S(stream);
  GridRows g{grid->x0, grid->y0, grid->h, grid->nx, grid->ny, row0, nrows};
  evaluate_grid(P, g, y_out, jac_out, S(stream));
  LENS_API_END
}

lens_status lens_ipm_map(lens_plan* plan, const lens_grid* grid, const lens_box* box, int npx,
                         int npy, int64_t max_cells_per_chunk, int bbox_cap_px, double* map_out,
                         lens_ipm_stats* stats, void* stream) {
  return lens_ipm_map_ex(plan, grid, box, npx, npy, max_cells_per_chunk, bbox_cap_px, 0, 0,
                         map_out, stats, stream);
}

lens_status lens_ipm_map_refined(lens_plan* plan, const lens_grid* grid, const lens_box* box,
                                 int npx, int npy, int64_t max_cells_per_chunk, int bbox_cap_px,
                                 int refine_levels, double* map_out, lens_ipm_stats* stats,
                                 void* stream) {
  return lens_ipm_map_ex(plan, grid, box, npx, npy, max_cells_per_chunk, bbox_cap_px,
                         refine_levels, 0, map_out, stats, stream);
}

lens_status lens_ipm_map_ex(lens_plan* plan, const lens_grid* grid, const lens_box* box, int npx,
                            int npy, int64_t max_cells_per_chunk, int bbox_cap_px,
                            int refine_levels, unsigned flags, double* map_out,
                            lens_ipm_stats* stats, void* stream) {
  LENS_API_BEGIN
  need(plan != nullptr, "plan is NULL");
  need((flags & ~(unsigned)(LENS_MAP_FUSED | LENS_MAP_SEPARATE)) == 0 &&
           flags != (LENS_MAP_FUSED | LENS_MAP_SEPARATE),
       "flags: LENS_MAP_FUSED or LENS_MAP_SEPARATE (or 0)");
  need(refine_levels >= 0 && refine_levels <= 16, "refine_levels must be in 0..16");
  need(refine_levels == 0 || bbox_cap_px > 0, "refinement needs a cap (bbox_cap_px > 0)");
  Plan& P = plan->P;
  check_grid(P, grid);
  need(!(flags & LENS_MAP_FUSED) || P.prec == LENS_FP32_BULK,
       "the fused map path needs a float32-bulk plan");
  const bool fused = (flags & LENS_MAP_FUSED) ||
                     (!(flags & LENS_MAP_SEPARATE) && P.prec == LENS_FP32_BULK && kFusedDefault);
  need(box != nullptr && map_out != nullptr, "box or map_out is NULL");
  need(npx >= 1 && npy >= 1 && (int64_t)npx * npy < (1ll << 31), "npx, npy must be >= 1 with npx*npy < 2^31");
  need(grid->nx < (1ll << 30), "grid nx must be below 2^30");
  need(std::isfinite(box->u0) && std::isfinite(box->u1) && std::isfinite(box->v0) &&
           std::isfinite(box->v1) && box->u1 > box->u0 && box->v1 > box->v0,
       "map window must be finite with u1 > u0, v1 > v0");
  need(max_cells_per_chunk >= 0 && bbox_cap_px >= 0, "chunk size and cap must be >= 0");
  cudaStream_t s = S(stream);
  P.da.stream = s;
  const int64_t nx = grid->nx, ny = grid->ny;
  int64_t max_cells = max_cells_per_chunk;
  if (max_cells == 0) {
    size_t fr = 0, tot = 0;
    LENS_CUDA(cudaMemGetInfo(&fr, &tot));
    // 16 B per corner + 4 B queue slot per cell, within a quarter of free memory
    max_cells = (int64_t)std::min<double>((double)fr / 4.0 / 20.0, (double)(1ll << 30));
  }
  max_cells = std::min<int64_t>(max_cells, 1ll << 30);
  // The float32 accumulators are flushed into the float64 map once about
  // kFlushCellsPerPixel cells per map pixel have entered them, so a pixel
  // sums a bounded number of float32 increments whatever the grid size
  // (a pixel under n equal increments drifts by up to ~n 2^-25 relative).
  constexpr int64_t kFlushCellsPerPixel = 64;
  const int64_t flush_cells = std::min<int64_t>(kFlushCellsPerPixel * npx * npy, 1ll << 30);
  max_cells = std::min(max_cells, flush_cells);
  int64_t rows = std::max<int64_t>(1, max_cells / nx);
  rows = std::min<int64_t>(rows, ny);
  need(rows * nx <= (1ll << 30) || rows == 1, "grid rows too wide for one chunk");

  IpmParams ip{};
  const double du = (box->u1 - box->u0) / npx, dv = (box->v1 - box->v0) / npy;
  ip.u0 = box->u0; ip.v0 = box->v0;
  ip.inv_du = 1.0 / du; ip.inv_dv = 1.0 / dv;
  ip.a_cell = grid->h * grid->h;
  ip.s_star = du * dv;
  ip.scale = ip.a_cell / ip.s_star;
  ip.npx = npx; ip.npy = npy; ip.cap = bbox_cap_px;

  Scratch corners(&P.da, sizeof(PixCorner) * (size_t)(rows + 1) * (size_t)(nx + 1));
  Scratch queue(&P.da, sizeof(int) * (size_t)rows * (size_t)nx + sizeof(int) * 4);
  Scratch sdev(&P.da, sizeof(double) * 16);
  // the map accumulates in float32 (increments are O(1) and a pixel receives
  // ~mu n_0 of them; float32 keeps ~1e-6 relative) and is written out in
  // float64 once at the end, so no float64 conversion runs per increment
  Scratch map32(&P.da, sizeof(float) * (size_t)npx * (size_t)npy);
  // whole-pixel runs of large cells enter as +v / -v at the ends of the run
  // in a per-row difference array, prefix-summed into the map at the end
  Scratch rowdiff(&P.da, sizeof(float) * ((size_t)npx + 1) * (size_t)npy);
  int* qcount = queue.as<int>() + (size_t)rows * (size_t)nx;
  // refinement: the grid cells of a chunk over the cap, then per level
  Scratch rq0(&P.da, refine_levels > 0 ? sizeof(int) * ((size_t)rows * (size_t)nx + 2) : 0);
  int* rq0count = refine_levels > 0 ? rq0.as<int>() + (size_t)rows * (size_t)nx : nullptr;
  int64_t refined = 0;
  LENS_CUDA(cudaMemsetAsync(map32.p, 0, map32.bytes, s));
  LENS_CUDA(cudaMemsetAsync(rowdiff.p, 0, rowdiff.bytes, s));
  LENS_CUDA(cudaMemsetAsync(sdev.p, 0, sdev.bytes, s));
  P.ev_clear();
  P.timing = true;
  P.work = sdev.as<double>() + 12;
  struct Reset {
    Plan& P;
    ~Reset() { P.timing = false; P.work = nullptr; P.ev_clear(); }
  } reset{P};
  std::vector<cudaEvent_t> ev;
  auto mark = [&]() {
    cudaEvent_t e;
    LENS_CUDA(cudaEventCreate(&e));
    LENS_CUDA(cudaEventRecord(e, s));
    ev.push_back(e);
  };
  int64_t chunks = 0, pending = 0;
  bool flushed = false;
  const long long l0 = launch_count();
  for (int64_t r0 = 0; r0 < ny; r0 += rows) {
    const int64_t nr = std::min<int64_t>(rows, ny - r0);
    if (pending > 0 && pending + nr * nx > flush_cells) {
      ipm_finish_map(map32.as<float>(), rowdiff.as<float>(), npx, npy, map_out, flushed, true, s);
      flushed = true;
      pending = 0;
    }
    GridRows g{grid->x0, grid->y0, grid->h, nx, ny, r0, nr + 1};
    if (rq0count) LENS_CUDA(cudaMemsetAsync(rq0count, 0, sizeof(int), s));
    if (fused) {
      // deflection and IPM in one kernel; only leaf-boundary corners reach
      // `corners`, for the seam cells mapped after it
      mark();
      evaluate_grid_fused(P, g, corners.as<PixCorner>(), ip, map32.as<float>(), rowdiff.as<float>(),
                          sdev.as<double>(), queue.as<int>(), qcount, rq0.as<int>(), rq0count, s);
      mark();
    } else {
      mark();
      evaluate_grid_pix(P, g, corners.as<PixCorner>(), ip, s);
      mark();
      ipm_accumulate(corners.as<PixCorner>(), nx, nr, ip, map32.as<float>(), rowdiff.as<float>(),
                     sdev.as<double>(), queue.as<int>(), qcount, rq0.as<int>(), rq0count, s,
                     &P.ev_ipm);
    }
    pending += nr * nx;
    ++chunks;
    if (refine_levels > 0) {
      // split the cells over the cap 2 x 2, level by level; the sub-cell
      // corner rays are not part of the grid's ray count
      double* work = P.work;
      P.work = nullptr;
      int np = 0;
      LENS_CUDA(cudaMemcpyAsync(&np, rq0count, sizeof(int), cudaMemcpyDeviceToHost, s));
      LENS_CUDA(cudaStreamSynchronize(s));
      Scratch parents_keep, org_keep;
      const int* parents = rq0.as<int>();
      const double2* org_in = nullptr;
      double hc = grid->h;
      for (int level = 1; level <= refine_levels && np > 0; ++level) {
        const bool more = level < refine_levels;
        Scratch org_out(&P.da, sizeof(double2) * 4 * (size_t)np);
        Scratch rq(&P.da, more ? sizeof(int) * (4 * (size_t)np + 2) : 0);
        int* rqc = more ? rq.as<int>() + 4 * (size_t)np : nullptr;
        if (rqc) LENS_CUDA(cudaMemsetAsync(rqc, 0, sizeof(int), s));
        ipm_refine(P, parents, np, org_in, grid->x0, grid->y0, r0, nx, hc, level, ip,
                   map32.as<float>(), rowdiff.as<float>(), sdev.as<double>(),
                   more ? rq.as<int>() : nullptr, rqc, org_out.as<double2>(), s, &P.ev_ipm);
        refined += np;
        pending += 4 * (int64_t)np;
        int next = 0;
        if (more) {
          LENS_CUDA(cudaMemcpyAsync(&next, rqc, sizeof(int), cudaMemcpyDeviceToHost, s));
          LENS_CUDA(cudaStreamSynchronize(s));
        }
        // this level's queue and corners feed the next one
        parents_keep = std::move(rq);
        org_keep = std::move(org_out);
        parents = parents_keep.as<int>();
        org_in = org_keep.as<double2>();
        np = next;
        hc *= 0.5;
      }
      P.work = work;
    }
  }
  ipm_finish_map(map32.as<float>(), rowdiff.as<float>(), npx, npy, map_out, flushed, false, s);
  mark();
  double hs[16];
  LENS_CUDA(cudaMemcpyAsync(hs, sdev.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
  LENS_CUDA(cudaStreamSynchronize(s));
  double msd = 0, msi = 0;
  for (size_t k = 0; k + 1 < ev.size(); ++k) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
    if (k % 2 == 0) msd += ms; else msi += ms;
  }
  for (auto e : ev) cudaEventDestroy(e);
  // every corner of every chunk must have been owned by exactly one leaf
  double expect_rays = 0;
  for (int64_t r0 = 0; r0 < ny; r0 += rows)
    expect_rays += (double)(std::min<int64_t>(rows, ny - r0) + 1) * (double)(nx + 1);
  if (hs[12] != expect_rays)
    fail(LENS_ECUDA, "internal: leaves covered " + std::to_string(hs[12]) + " of " +
                         std::to_string(expect_rays) + " grid rays");
  double mse = 0, msk = 0;
  for (auto& e : P.ev_eval) { float ms = 0; cudaEventElapsedTime(&ms, e.first, e.second); mse += ms; }
  for (auto& e : P.ev_ipm) { float ms = 0; cudaEventElapsedTime(&ms, e.first, e.second); msk += ms; }
  double msf = 0;
  for (auto& e : P.ev_fused) { float ms = 0; cudaEventElapsedTime(&ms, e.first, e.second); msf += ms; }
  if (stats) {
    stats->cells = (double)nx * (double)ny;
    stats->area_total = stats->cells * ip.a_cell;
    stats->area_in_map = ip.a_cell * hs[2];
    stats->area_outside = ip.a_cell * hs[3];
    stats->area_dropped = ip.a_cell * hs[6];
    stats->area_degenerate = ip.a_cell * hs[7];
    stats->cells_dropped = hs[4];
    stats->cells_degenerate = hs[5];
    stats->chunks = chunks;
    stats->ms_deflect = msd;
    stats->ms_ipm = msi;
    stats->rays = hs[12];
    stats->p2p_pairs = hs[13];
    stats->m2p_evals = hs[14];
    stats->ipm_updates = hs[8];
    stats->cells_queued = hs[9];
    stats->cells_ext = hs[10];
    stats->ms_eval_kernel = mse;
    stats->ms_ipm_kernel = msk;
    stats->launches = launch_count() - l0;
    stats->cells_refined = (double)refined;
    stats->fused = fused ? 1 : 0;
    stats->ms_fused_kernel = msf;
    stats->rays_evaluated = fused ? hs[15] : hs[12];
  }
  LENS_API_END
}

lens_status lens_deflect_adjoint(lens_plan* plan, const double* rays_xy, int64_t m,
                                 const double* grad_y, double* grad_xy, double* grad_m,
                                 double* grad_kg, void* stream) {
  LENS_API_BEGIN
  need(plan != nullptr, "plan is NULL");
  need(m >= 0, "m must be >= 0");
  need(m == 0 || (rays_xy && grad_y), "rays or grad_y is NULL");
  need(m < (int64_t)INT32_MAX, "too many rays in one call");
  Plan& P = plan->P;
  P.da.stream = S(stream);
  adjoint(P, rays_xy, m, grad_y, grad_xy, grad_m, grad_kg, S(stream));
  LENS_API_END
}

lens_status lens_direct_deflect(const double* stars_xy, const double* masses, int64_t n,
                                double kappa_s, double gamma, const double* rays_xy, int64_t m,
                                int prec, double* y_out, double* jac_out,
                                const lens_allocator* allocator, void* stream) {
  LENS_API_BEGIN
  need(n >= 0 && m >= 0, "sizes must be >= 0");
  need(prec == LENS_FP64 || prec == LENS_FP32_BULK, "prec must be LENS_FP64 or LENS_FP32_BULK");
  if (m == 0) return LENS_OK;
  need(rays_xy && y_out && (n == 0 || (stars_xy && masses)), "NULL buffer");
  DeviceAlloc da;
  da.stream = S(stream);
  if (allocator && allocator->alloc && allocator->free) { da.a = *allocator; da.custom = true; }
  direct_deflect(stars_xy, masses, n, kappa_s, gamma, rays_xy, m, prec, y_out, jac_out, da,
                 S(stream));
  LENS_API_END
}

lens_status lens_light_curve(const double* y, int64_t m, double w_ray, const double* samples,
                             int64_t ns, double sigma, double trunc, double* F_out, void* stream) {
  LENS_API_BEGIN
  need(m >= 0 && ns >= 0, "sizes must be >= 0");
  need(sigma > 0 && trunc > 0 && std::isfinite(sigma) && std::isfinite(trunc), "sigma, trunc must be > 0");
  if (ns == 0) return LENS_OK;
  need(F_out && samples && (m == 0 || y), "NULL buffer");
  light_curve(y, m, w_ray, samples, ns, sigma, trunc, F_out, S(stream));
  LENS_API_END
}

lens_status lens_light_curve_grad(const double* y, int64_t m, double w_ray, const double* samples,
                                  int64_t ns, double sigma, double trunc, const double* F,
                                  const double* T, double* grad_y_out, void* stream) {
  LENS_API_BEGIN
  need(m >= 0 && ns >= 0, "sizes must be >= 0");
  need(sigma > 0 && trunc > 0 && std::isfinite(sigma) && std::isfinite(trunc), "sigma, trunc must be > 0");
  if (m == 0) return LENS_OK;
  need(grad_y_out && y && (ns == 0 || (samples && F && T)), "NULL buffer");
  light_curve_grad(y, m, w_ray, samples, ns, sigma, trunc, F, T, grad_y_out, S(stream));
  LENS_API_END
}

lens_status lens_map_source(const double* map, int npx, int npy, double sigma_px, double trunc,
                            double* out, const lens_allocator* allocator, void* stream) {
  LENS_API_BEGIN
  need(map && out, "NULL buffer");
  need(map != out, "out may not alias map");
  need(npx >= 1 && npy >= 1 && (int64_t)npx * npy < (1ll << 31), "npx, npy must be >= 1 with npx*npy < 2^31");
  need(sigma_px > 0 && trunc > 0 && std::isfinite(sigma_px) && std::isfinite(trunc),
       "sigma_px, trunc must be finite and > 0");
  DeviceAlloc da;
  if (allocator) { da.a = *allocator; da.custom = true; }
  da.stream = S(stream);
  map_source(map, npx, npy, sigma_px, trunc, out, da, S(stream));
  LENS_API_END
}

lens_status lens_map_histogram(const double* values, int64_t n, double lo, double hi, int nbins,
                               int log_bins, int64_t* counts, void* stream) {
  LENS_API_BEGIN
  need(n >= 0, "n must be >= 0");
  need(counts && (n == 0 || values), "NULL buffer");
  need(nbins >= 1 && nbins <= 8192, "nbins must be in 1..8192");
  need(std::isfinite(lo) && std::isfinite(hi) && hi > lo, "need finite lo < hi");
  map_histogram(values, n, lo, hi, nbins, log_bins ? 1 : 0, counts, S(stream));
  LENS_API_END
}

lens_status lens_map_track(const double* map, int npx, int npy, const lens_box* box,
                           const double* positions, int64_t ns, double* out, void* stream) {
  LENS_API_BEGIN
  need(ns >= 0, "ns must be >= 0");
  need(box && map && (ns == 0 || (positions && out)), "NULL buffer");
  need(npx >= 1 && npy >= 1 && (int64_t)npx * npy < (1ll << 31), "npx, npy must be >= 1 with npx*npy < 2^31");
  need(std::isfinite(box->u0) && std::isfinite(box->u1) && std::isfinite(box->v0) &&
           std::isfinite(box->v1) && box->u1 > box->u0 && box->v1 > box->v0,
       "map window must be finite with u1 > u0, v1 > v0");
  const double b[4] = {box->u0, box->u1, box->v0, box->v1};
  map_track(map, npx, npy, b, positions, ns, out, S(stream));
  LENS_API_END
}

lens_status lens_find_images(const double* y, const lens_grid* grid, double beta1, double beta2,
                             int64_t max_out, double* out, int64_t* cells, int64_t* n_found,
                             void* stream) {
  LENS_API_BEGIN
  need(y && grid && n_found, "NULL buffer");
  need(max_out >= 0 && (max_out == 0 || (out && cells)), "max_out must be >= 0 with buffers");
  need(grid->nx >= 1 && grid->ny >= 1 && grid->nx < (1ll << 31) && grid->ny < (1ll << 31),
       "grid must have 1 <= nx, ny < 2^31");
  need(std::isfinite(grid->x0) && std::isfinite(grid->y0) && std::isfinite(grid->h) && grid->h > 0,
       "grid origin and spacing must be finite with h > 0");
  need(std::isfinite(beta1) && std::isfinite(beta2), "beta must be finite");
  DeviceAlloc da;
  da.stream = S(stream);
  *n_found = find_images(y, grid->nx, grid->ny, grid->x0, grid->y0, grid->h, beta1, beta2, max_out,
                         out, cells, da, S(stream));
  LENS_API_END
}

lens_status lens_source_image(const double* y, int64_t m, double beta1, double beta2, double sigma,
                              double* out, void* stream) {
  LENS_API_BEGIN
  need(m >= 0, "m must be >= 0");
  need(m == 0 || (y && out), "NULL buffer");
  need(std::isfinite(beta1) && std::isfinite(beta2), "beta must be finite");
  need(std::isfinite(sigma) && sigma > 0, "sigma must be finite and > 0");
  source_image(y, m, beta1, beta2, sigma, out, S(stream));
  LENS_API_END
}

}  // extern "C"
