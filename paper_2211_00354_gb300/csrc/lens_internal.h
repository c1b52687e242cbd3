// lens_internal.h -- host-side plumbing shared by the liblens translation units:
// the plan object, status/exception handling, device allocation through the
// caller's allocator, host-side fault injection and launch checking.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lens.h"
#include "cx.cuh"

namespace lens {

// Internal failures are C++ exceptions that every extern "C" entry point
// converts to a lens_status (nothing crosses the ABI).
struct Error {
  lens_status status;
  std::string msg;
};

[[noreturn]] void fail(lens_status st, const std::string& msg);
void set_last_error(const std::string& msg);

void check_cuda(cudaError_t e, const char* what);
// Called after every kernel launch: counts launches (LENS_FAULT=launch@K)
// and turns a launch error into LENS_ECUDA.
void after_launch(const char* name);
// Counts allocations (LENS_FAULT=alloc@K); throws LENS_EFAULT_INJECTED when due.
void fault_point_alloc();
// kernels launched so far by this process (through LENS_LAUNCHED)
long long launch_count();

#define LENS_CUDA(call) ::lens::check_cuda((call), #call)
#define LENS_LAUNCHED(name) ::lens::after_launch(name)

// Device memory provider: the caller's lens_allocator, or cudaMallocAsync.
struct DeviceAlloc {
  lens_allocator a{};
  bool custom = false;
  cudaStream_t stream = nullptr;
  void* alloc(size_t bytes);
  void release(void* p);
};

// Scoped scratch buffer (freed, stream-ordered, when it leaves scope).
struct Scratch {
  DeviceAlloc* da = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  Scratch() = default;
  Scratch(DeviceAlloc* d, size_t b) : da(d), bytes(b) { p = b ? d->alloc(b) : nullptr; }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  Scratch(Scratch&& o) noexcept : da(o.da), p(o.p), bytes(o.bytes) { o.p = nullptr; }
  Scratch& operator=(Scratch&& o) noexcept {
    if (this != &o) { reset(); da = o.da; p = o.p; bytes = o.bytes; o.p = nullptr; }
    return *this;
  }
  ~Scratch() { reset(); }
  void reset() { if (p && da) da->release(p); p = nullptr; }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

constexpr int kMaxDepth = 28;   // quadtree levels below the root (56-bit keys)
constexpr int kMaxOrder = 64;   // expansion order cap

// Float32 evaluation kernel geometry (eval32.cu): threads per CTA, rays per thread.
constexpr int kEval32Threads = 128;
constexpr int kEval32Rpt = 4;

// Per active leaf, float64 constants formed once per plan (eval32.cu).
struct LeafPlan {
  double cx, cy;  // leaf centre
  double K1, K2;  // a c1 - b0_1 and b c2 + b0_2 (lens equation at the centre)
  float ir, r;    // 1/r and r (half-side)
};
// Per active leaf and call on the grid path (eval32.cu).
struct LeafGrid {
  ff bx, by;      // offset of the leaf's first grid ray from its centre
  ff U1f, V1f;    // fractional part of the centre's pixel reference (map path)
  int U1i, V1i;   // integer part
  int far;        // the reference lies beyond 2^30 pixels
  int pad;
  // grid units: the grid point nearest the centre (clamped into the grid) is
  // the leaf's origin, the same for every band of rows the grid is cut into
  ff rx, ry;      // its offset from the centre
  int ri, rj;     // the first grid ray's index minus its index
};

// Host-built float64 tables for one order p (device copies owned by the plan).
struct FmmTables {
  int p = 0, ldb = 0;
  double* binom = nullptr;   // C(n, k), n < 2p+2, k < p+2: binom[n*ldb + k]
  double2* m2m = nullptr;    // [4][p+1][p+1]: row l, col k (k <= l)
  double2* l2l = nullptr;    // [4][p+1][p+1]: row j, col l (l >= j)
  double2* upow = nullptr;   // [49][p+2]: u^k for offset (dx,dy) in [-3,3]^2
  double2* wpow = nullptr;   // [p+1]: ((1+i)/2)^k, exact in float64
};

struct Plan {
  int device = 0;
  DeviceAlloc da;
  std::vector<void*> owned;  // plan-lifetime device allocations
  int64_t device_bytes = 0;

  int64_t n = 0;
  int p = 0, leaf = 0, prec = 0, depth = kMaxDepth;
  bool equal_mass = false;  // every star has mass mass0
  double mass0 = 0.0;
  double kappa_s = 0, gamma = 0;
  double root_lo[2] = {0, 0}, root_size = 1;
  bool has_target = false;
  double target[4] = {0, 0, 0, 0};

  int nlevels = 0;                     // levels 0 .. nlevels-1 hold boxes
  std::vector<int64_t> level_off;      // box ids of level l: [level_off[l], level_off[l+1])
  int64_t nb = 0;

  // sorted stars (Morton order)
  double2* spos = nullptr;
  double* smass = nullptr;
  uint32_t* sidx = nullptr;            // sorted slot -> caller index
  uint64_t* skey = nullptr;

  // boxes (structure of arrays, level-major, Morton order within a level)
  int* box_start = nullptr;
  int* box_count = nullptr;
  int* box_child = nullptr;            // first of 4 children, -1 for a leaf
  int* box_parent = nullptr;
  int* box_level = nullptr;
  int* box_ix = nullptr;
  int* box_iy = nullptr;
  uint64_t* box_code = nullptr;        // Morton code of (ix, iy) at its level
  uint8_t* box_active = nullptr;

  // active boxes (meet the target region), level-major
  int64_t n_active = 0, n_active_leaves = 0;
  int* active = nullptr;               // active box ids
  std::vector<int64_t> active_level_off;
  int* active_leaves = nullptr;        // active leaf ids
  int* box_aidx = nullptr;             // box id -> active index, -1 if inactive
  int* box_lidx = nullptr;             // box id -> active-leaf index, -1 otherwise

  // interaction lists, CSR over the active list index
  int64_t nV = 0, nX = 0, nU = 0, nW = 0, u_stars = 0;
  // (all four lists are indexed by the active index; U and W are empty for
  //  internal boxes)
  int64_t* V_off = nullptr; int* V_list = nullptr;
  int64_t* X_off = nullptr; int* X_list = nullptr;
  int64_t* U_off = nullptr; int* U_list = nullptr;
  int64_t* W_off = nullptr; int* W_list = nullptr;

  // expansions: (p+1) complex coefficients per box, scaled (see fmm.cu)
  double2* M = nullptr;
  double2* L = nullptr;
  int* p2m_list = nullptr;  // non-empty leaves sorted by star count (nb slots)
  int* p2m_bins = nullptr;  // 2 (leaf_size + 1): counts and offsets per star count
  FmmTables tab;

  // float32-bulk evaluation data (eval32_prepare)
  LeafPlan* f_leaf = nullptr;   // per active leaf
  float2* f_L = nullptr;        // per active leaf, (p+1) local coefficients
  float2* f_M = nullptr;        // per box, (p+1) multipole coefficients (far W boxes filled)
  // near field of every active leaf k (its U-list leaves plus the W boxes
  // small enough for P2P): the stars as float-float offsets from the leaf
  // centre (f_ust / f_um from f_uoff[k]); the far W boxes left to M2P
  // (f_wlist / f_wgeo from f_woff[k]); per-leaf counts of near stars
  // (f_ncnt) and far W boxes (f_wcnt) for the work counters
  float4* f_ust = nullptr;
  float* f_um = nullptr;
  int64_t* f_uoff = nullptr;
  int64_t* f_woff = nullptr; int* f_wlist = nullptr;
  int64_t f_nw = 0;             // far W entries in f_wlist
  float4* f_wgeo = nullptr;     // per far W entry: centre offset from the leaf centre, radius
  int64_t* f_ncnt = nullptr; int64_t* f_wcnt = nullptr;

  double ms_build = 0;
  int64_t build_launches = 0;

  // Once the boxes exist (ev_boxes), P2M and M2M run on a low-priority
  // stream of the plan (ev_up marks their end) while the interaction lists
  // are formed on a high-priority one (ev_lists); the downward pass follows
  // both on the high-priority stream, the float32 near-field staging follows
  // the lists on the caller's stream (ev_tree), and the float32 copies of
  // the expansions follow both (ev_fmm marks the end).  Work that reads M or
  // L waits on ev_fmm (wait_expansions); work that needs only the tree waits
  // on ev_tree.
  cudaStream_t fmm_stream = nullptr, up_stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_boxes = nullptr, ev_tree = nullptr, ev_fmm = nullptr;
  cudaEvent_t ev_up = nullptr, ev_lists = nullptr;
  // host copies of the translation tables, alive until their copies have run
  std::vector<double> tab_host;
  // around the far-field launch (M2L over V, P2L over X) on the plan's stream
  cudaEvent_t ev_far0 = nullptr, ev_far1 = nullptr;
  bool build_timed = false;

  // per-active-index count of stars in the U list (work accounting)
  int64_t* ustar_cnt = nullptr;
  // optional kernel timing and work counters (lens_ipm_map turns them on)
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_eval, ev_ipm, ev_fused;
  double* work = nullptr;  // device [4]: rays, p2p pairs, m2p evals, spare
  void ev_clear() {
    for (auto& e : ev_eval) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto& e : ev_ipm) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto& e : ev_fused) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    ev_eval.clear();
    ev_ipm.clear();
    ev_fused.clear();
  }

  void* dalloc(size_t bytes) {
    void* p = da.alloc(bytes);
    owned.push_back(p);
    device_bytes += (int64_t)bytes;
    return p;
  }
  template <class T> T* dalloc_n(size_t count) {
    return static_cast<T*>(dalloc(count * sizeof(T) + (count == 0 ? 16 : 0)));
  }
  double half_side(int level) const { return root_size / (double)(2ull << level); }
};

// ---- launchers (defined in the .cu files) --------------------------------
void direct_deflect(const double* stars, const double* masses, int64_t n,
                    double ks, double g, const double* rays, int64_t m, int prec,
                    double* y, double* jac, DeviceAlloc& da, cudaStream_t s);

// Stable LSD sort of (keys, vals) by key bits [lo_bit, bits), 8 bits a pass.
void radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int bits,
                    DeviceAlloc& da, cudaStream_t s, int lo_bit = 0);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, DeviceAlloc& da,
                        cudaStream_t s);
// host[i] = *addrs[i] (device int64 values, n <= kMaxPick): one small kernel,
// one copy and one synchronisation instead of a round trip per value (a
// device-to-pageable copy returns only when it is done)
constexpr int kMaxPick = 64;
void read_i64(const int64_t* const* addrs, int n, int64_t* host, DeviceAlloc& da, cudaStream_t s);

// Tree build in two halves: the boxes (bounds, keys, sort, splits: all the
// upward pass needs), then the active boxes and the interaction lists.
void tree_build_boxes(Plan& P, const double* stars, const double* masses, cudaStream_t s);
void tree_build_lists(Plan& P, cudaStream_t s);
void fmm_tables(Plan& P, cudaStream_t s);
// expansion buffers (M, L, P2M leaf order), allocated on the caller's stream
// before the expansions are handed to the plan's own stream
void fmm_alloc(Plan& P);
void fmm_p2m(Plan& P, cudaStream_t s);
void fmm_m2m(Plan& P, cudaStream_t s);
void fmm_downward(Plan& P, cudaStream_t s);

struct GridRows {  // a band of corner rows of a grid
  double x0, y0, h;
  int64_t nx, ny;   // cells (corners nx+1 by ny+1)
  int64_t row0, nrows;
};
void evaluate_grid(Plan& P, const GridRows& g, double* y, double* jac, cudaStream_t s);
void evaluate_rays(Plan& P, const double* rays, int64_t m, double* y, double* jac,
                   cudaStream_t s);
// Rays bucketed by active leaf: perm (ray ids in leaf order), off (per leaf,
// CSR into perm) and toff (per leaf, first tile of `tile` rays).
struct RayBuckets {
  Scratch perm, off, toff;
  int64_t total = 0;  // tiles
};
void bucket_rays(Plan& P, const double* rays, int64_t m, int tile, RayBuckets& B, cudaStream_t s);

struct IpmParams {
  double u0, v0, inv_du, inv_dv;  // source-plane window origin, inverse pixel size
  double scale;                   // A_cell / S* (map increment per unit fraction)
  double a_cell, s_star;          // cell area h^2, pixel area S*
  int npx, npy, cap;
};
// A deflected corner in map-pixel coordinates: u = iu + fu, fu in [0, 1];
// iu == iv == INT32_MAX marks a corner farther than 2^30 pixels.
struct __align__(16) PixCorner {
  int iu; float fu; int iv; float fv;
};
void evaluate_grid_pix(Plan& P, const GridRows& g, PixCorner* out, const IpmParams& ip,
                       cudaStream_t s);
// map32: float32 accumulation map (npy x npx); rowdiff: float32 per-row
// difference array (npy x (npx + 1)) for whole-pixel runs of large cells.
// rq / rqcount: with refinement, the cells over the cap are queued there
// instead of dropped (NULL: dropped).
void ipm_accumulate(const PixCorner* yc, int64_t nx, int64_t nrows_cells, const IpmParams& ip,
                    float* map32, float* rowdiff, double* stats_dev, int* queue, int* qcount,
                    int* rq, int* rqcount, cudaStream_t s,
                    std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev);
// ipm_accumulate over a list of n cells (ids j * nx + i into yc's grid)
void ipm_accumulate_list(const PixCorner* yc, int64_t nx, const int* list, int64_t n,
                         const IpmParams& ip, float* map32, float* rowdiff, double* stats_dev,
                         int* queue, int* qcount, int* rq, int* rqcount, cudaStream_t s,
                         std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev);
// One refinement level: each of the np queued cells (cells of the chunk
// starting at grid row grow0 when org_in is NULL, else sub-cells with
// lower-left corners org_in[]) of side h is split into 2 x 2 sub-cells of
// side h/2, whose corners are deflected (the plan's ray path) and mapped with
// weight 4^-level.  Sub-cells over the cap go to rq_next (NULL: dropped);
// org_out receives the 4 np sub-cell corners.  Returns the sub-cells mapped.
int64_t ipm_refine(Plan& P, const int* parents, int64_t np, const double2* org_in, double gx0,
                   double gy0, int64_t grow0, int64_t gnx, double h, int level,
                   const IpmParams& ip, float* map,
                   float* rowdiff, double* stats_dev, int* rq_next, int* rqcount_next,
                   double2* org_out, cudaStream_t s,
                   std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev);
// float32 evaluation data that needs only the tree (leaf geometry, staged
// near-field stars, far W boxes), and the part that needs the expansions
// (constants of the lens equation per leaf, float32 copies of L and M);
// eval32_alloc reserves both before the expansions start
void eval32_alloc(Plan& P);
void eval32_prepare_tree(Plan& P, cudaStream_t s);
void eval32_prepare_expansions(Plan& P, cudaStream_t s);
// make stream s wait for the plan's expansions (which implies its tree), or
// for its tree and tree-only data alone
void wait_expansions(Plan& P, cudaStream_t s);
void wait_tree(Plan& P, cudaStream_t s);
void eval32_grid(Plan& P, const GridRows& g, const int64_t* rect, const int2* tile_leaf,
                 int64_t total, double* y, double* jac, PixCorner* pix, const IpmParams* ip,
                 cudaStream_t s);
void eval32_rays(Plan& P, const double* rays, const int64_t* off, const int* perm,
                 const int2* tile_leaf, int64_t total, double* y, double* jac, cudaStream_t s);
// The fused deflection + IPM path (eval32.cu, float32-bulk plans).  A work
// item is a rectangle of one leaf's grid corners: w x h corners from corner
// (ci, cj) counted from the leaf's first ray; the items of a leaf overlap by
// one corner row / column, which both evaluate from the leaf's data to the
// same bits.  The kernel maps every cell whose four corners lie in its item;
// the cells on a leaf's last corner row or column (their other corners
// belong to neighbouring leaves) are mapped afterwards from the corners on
// leaf boundaries, the only ones written to device memory (`edge`, in the
// chunk's grid layout).  Returns the seam cells (ids j * nx + i in the chunk)
// and their count.
struct FuseItem {
  int leaf;    // active-leaf index
  int ci, cj;  // first corner of the item, relative to the leaf's first ray
  int w, h;    // corners in the item
};
struct IpmArgs;
void ipm_prepare(IpmArgs& A);
Scratch eval32_fused(Plan& P, const GridRows& g, const int64_t* rect, PixCorner* edge,
                     const IpmParams& ip, float* map32, float* rowdiff, double* stats_dev, int* rq,
                     int* rqcount, int64_t& nseam, cudaStream_t s);
void evaluate_grid_fused(Plan& P, const GridRows& g, PixCorner* edge, const IpmParams& ip,
                         float* map32, float* rowdiff, double* stats_dev, int* queue, int* qcount,
                         int* rq, int* rqcount, cudaStream_t s);
// map = map32 + row-wise prefix sums of rowdiff (mapfinish.cu): `clear` (a
// flush between chunks) keeps the sum in map's slots as float-float pairs
// and zeroes map32 and rowdiff; otherwise float64 is written, the pairs
// added first with `accumulate`
void ipm_finish_map(float* map32, float* rowdiff, int npx, int npy, double* map, bool accumulate,
                    bool clear, cudaStream_t s);
// map consumers (mapops.cu): Gaussian finite source, histogram, track
void map_source(const double* map, int npx, int npy, double sigma_px, double trunc, double* out,
                DeviceAlloc& da, cudaStream_t s);
void map_histogram(const double* v, int64_t n, double lo, double hi, int nbins, int log_bins,
                   int64_t* counts, cudaStream_t s);
void map_track(const double* map, int npx, int npy, const double box[4], const double* pos,
               int64_t ns, double* out, cudaStream_t s);
// a pair of recorded events bracketing work on a stream
std::pair<cudaEvent_t, cudaEvent_t> event_pair_begin(cudaStream_t s);
void event_pair_end(std::pair<cudaEvent_t, cudaEvent_t>& e, cudaStream_t s);

void adjoint(Plan& P, const double* rays, int64_t m, const double* gy,
             double* gxy, double* gm, double* gkg, cudaStream_t s);

void light_curve(const double* y, int64_t m, double w, const double* smp, int64_t ns,
                 double sigma, double trunc, double* F, cudaStream_t s);
void light_curve_grad(const double* y, int64_t m, double w, const double* smp,
                      int64_t ns, double sigma, double trunc, const double* F,
                      const double* T, double* gy, cudaStream_t s);

// grid size helper: blocks of `threads` covering n, capped
inline unsigned grid_for(int64_t n, int threads, int64_t cap = (1ll << 31) - 1) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace lens
