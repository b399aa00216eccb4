// gl_api.cu -- kernels and the C-ABI (include/gl.h) of the oblate-transit library.
//
// One B300 (sm_103a), one process.  Kernels:
//   gl_setup_kernel    one thread per parameter set: projected ellipse (Sec. 2,
//                      Eqs. dx, dy1, dy2; Appendix A), LD basis, orbit constants,
//                      transit window (FP64)
//   gl_curve_kernel    one thread per exposure: window test, then per
//                      sub-exposure Kepler solve (FP64), overlap class, Green's
//                      theorem quadrature (R = double or float) and the FP64
//                      exposure mean
//   gl_sky_kernel      geometry-level flux for given sky positions
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <array>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/gl.h"
#include "gl_math.cuh"

using gl::NodeRule;
using gl::SetConst;

namespace {

// status bits accumulated on the device
enum : int { kStatusInvalidSet = 1, kStatusBadOffsets = 2, kStatusTimeout = 4, kStatusOverflow = 8 };
// NVTX range over a scope (shown by profilers on the host timeline; a no-op
// when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Boundaries of a light-curve step at which profiling mode 2 records events
// inside the step graph: before the constants, then after each kernel.
enum : int { kMarkStart = 0, kMarkSetup, kMarkWindow, kMarkExposures, kMarkItems, kMarkSums,
             kMarks };

// quadrature orders: FP64 path and FP32C path
constexpr int kNodes64 = 32;
constexpr int kNodes64Wide = 48;   // FP64 order for large, strongly flattened shapes
constexpr int kNodes32 = 20;

// item pipeline workspace: at most this many sub-exposure items per call by
// default; per item 3 positions + deficit (FP64 sizing) + set + queue slot +
// record index, and a record (at most one per item: output index, first item,
// count, set, flags, tau, midpoint state); plus three ints per exposure for
// the kept-exposure list and the overflow list
constexpr int64_t kItemMaxDefault = 1LL << 23;
constexpr size_t kItemBytes = 4 * sizeof(double) + 6 * sizeof(int);

__constant__ NodeRule<double> c_rule64;
__constant__ double c_inv_n[65];   // 1 / n for n = 1..64 (entry 0 unused)

// Exposure flux from S, the FP64 sum of its n sub-exposure deficits: the mean of
// 1 - deficit, 1 - S / n (one FMA with 1/n from a table; every path of the light
// curve ends here, so they agree to the bit).
__device__ __forceinline__ double exposure_mean(double S, int n) {
  const double inv = n <= 64 ? c_inv_n[n] : 1.0 / (double)n;
  return fma(-S, inv, 1.0);
}
__constant__ NodeRule<double> c_rule64_wide;
__constant__ NodeRule<float> c_rule32;                 // default order (kNodes32)
// orders the autotuner may choose for the FP32C light-curve kernel
constexpr int kTuneNodes[4] = {16, 20, 24, 28};
constexpr int kRuleDefault = 1;   // 20 nodes
__constant__ NodeRule<float> c_rule32_tuned[4];

template <typename R> __device__ __forceinline__ const NodeRule<R>& rule();
template <> __device__ __forceinline__ const NodeRule<double>& rule<double>() { return c_rule64; }
template <> __device__ __forceinline__ const NodeRule<float>& rule<float>() { return c_rule32; }

// Quadrature rule of parameter set c: FP64 (32 nodes, 48 for shapes with a
// raised FP32 order), or the FP32 order `base` (index into c_rule32_tuned)
// raised to the set's least order for its shape.
template <typename R>
__device__ __forceinline__ const NodeRule<R>& set_rule(const SetConst& c, int base);
template <>
__device__ __forceinline__ const NodeRule<double>& set_rule<double>(const SetConst& c, int) {
  // shapes that need more FP32 nodes also need more FP64 ones: 32 nodes leave
  // errors up to 3e-10 near tangency there, 48 keep them below 1e-12
  return c.rule_min > 0 ? c_rule64_wide : c_rule64;
}
template <>
__device__ __forceinline__ const NodeRule<float>& set_rule<float>(const SetConst& c, int base) {
  return c_rule32_tuned[base > c.rule_min ? base : c.rule_min];
}

// ------------------------------------------------------------------ kernels
// Programmatic dependent launch: the item pipeline's kernels after the setup
// kernel are launched with programmatic stream serialisation, so a kernel's CTAs
// are dispatched as its predecessor's CTAs exit rather than after the
// predecessor's completion has been signalled, and each waits in pdl_wait, before
// it touches memory, until the predecessor has completed and its writes are
// visible (a no-op for a kernel launched without the attribute).  No kernel
// triggers its successor early: successors resident beside a running kernel
// measured slower than the saved launch latency.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct ParamPtrs {
  const double *t0, *period, *a_rs, *b, *ecc, *omega, *k, *f, *eta, *xi, *u1, *u2;
  const double *g, *zeta;   // optional triaxial shape (NULL: oblate)
  const double* exptime;
  const int32_t* nsuper;
  int32_t nsuper_all;
};

// 32 sets per 128-thread block, one role per warp, so that the four FP64
// instruction streams run on four SM sub-partitions at once (an FP64 warp
// instruction costs the same whether one lane or 32 are active).
//   stage 1: warps 0-2 compute sin and cos of omega, xi and eta, warp 3 the cube
//            root of 1 - f, one set per lane
//   stage 2: warp 0 the orbit and validity, warp 1 the projected ellipse and
//            the exposure fields, warp 2 the transit window, warp 3 the limb
//            darkening, each writing its own fields of the set's constants; warp
//            0 then sets the flags.  (Stamped per warp with the exposure fields
//            in warp 2, the stage took 4.1, 2.7, 4.7 and 4.1 us in warps 0-3.)
__global__ void __launch_bounds__(128) gl_setup_kernel(ParamPtrs p, int64_t n_sets,
                                                       const int64_t* offsets, int64_t n_total,
                                                       SetConst* sets, int* status,
                                                       unsigned long long* zero, int n_zero) {
  __shared__ double sh_s[4][32], sh_c[4][32], sh_cb[32];
  __shared__ int sh_win[32], sh_tay[32], sh_valid[32];
  const int lane = threadIdx.x & 31, role = threadIdx.x >> 5;
  if (zero)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_zero; i += gridDim.x * blockDim.x)
      zero[i] = 0ull;
  const int64_t s = (int64_t)blockIdx.x * 32 + lane;
  const bool live = s < n_sets;
  if (role < 3) {
    double v0 = 0.0, v1 = 1.0;
    const double ang = live ? (role == 0 ? p.omega[s] : role == 1 ? p.xi[s] : p.eta[s]) : 0.0;
    if (isfinite(ang)) gl::sincos_setup(ang, &v0, &v1);
    sh_s[role][lane] = v0;
    sh_c[role][lane] = v1;
  } else {
    // cube root of (1 - f)(1 - g) and, for a triaxial shape, sin and cos of zeta
    const double f = live ? p.f[s] : 0.0;
    const double g = (live && p.g) ? p.g[s] : 0.0;
    const double q = (1.0 - f) * (1.0 - g);
    sh_cb[lane] = (isfinite(q) && q > 0.0) ? gl::cbrt_setup(q) : 1.0;
    double v0 = 0.0, v1 = 1.0;
    const double zeta = (live && p.zeta) ? p.zeta[s] : 0.0;
    if (p.g && isfinite(zeta)) gl::sincos_setup(zeta, &v0, &v1);
    sh_s[3][lane] = v0;
    sh_c[3][lane] = v1;
  }
  __syncthreads();
  const double cb = sh_cb[lane];
  int orbit_ok = 0;
  if (live) {
    SetConst* c = sets + s;
    // four FP64 chains of similar length, one per warp
    if (role == 0) {
      orbit_ok = gl::set_orbit(p.t0[s], p.period[s], p.a_rs[s], p.b[s], p.ecc[s], sh_s[0][lane],
                               sh_c[0][lane], c);
      gl::set_kepler(c);   // (meaningless for an invalid orbit; such sets are never used)
    } else if (role == 1) {
      const double g = p.g ? p.g[s] : 0.0, f = p.f[s];
      if (g != 0.0)
        gl::set_shape_triaxial(p.k[s], f, g, cb, sh_s[3][lane], sh_c[3][lane],
                               sh_s[2][lane], sh_c[2][lane], sh_s[1][lane], sh_c[1][lane], c);
      else
        gl::set_shape(p.k[s], f, cb, sh_c[2][lane], sh_s[1][lane], sh_c[1][lane], c);
      const double period = p.period[s], invP = gl::rcp64(period);
      sh_tay[lane] = gl::set_exposure(p.t0[s], period, p.a_rs[s], p.ecc[s], 2.0 * gl::kPi * invP, invP,
                                      p.exptime[s], p.nsuper ? p.nsuper[s] : p.nsuper_all, c);
    } else if (role == 2) {
      const double period = p.period[s], invP = gl::rcp64(period);
      sh_win[lane] = gl::set_window(p.t0[s], period, p.a_rs[s], p.ecc[s], p.omega[s],
                                    gl::set_req(p.k[s], cb), 2.0 * gl::kPi * invP, invP,
                                    p.exptime[s], p.nsuper ? p.nsuper[s] : p.nsuper_all, c);
    } else {
      gl::set_ld(p.u1[s], p.u2[s], c);
      const double g = p.g ? p.g[s] : 0.0, f = p.f[s];
      const double cax = p.k[s] * gl::rcp64(cb);   // c = k ((1 - f)(1 - g))^(-1/3)
      gl::set_body(cax * (1.0 - f), cax * (1.0 - g), cax, sh_s[3][lane], sh_c[3][lane],
                   sh_s[2][lane], sh_c[2][lane], sh_s[1][lane], sh_c[1][lane], c);
      const int ns = p.nsuper ? p.nsuper[s] : p.nsuper_all;
      const double zeta = p.zeta ? p.zeta[s] : 0.0;
      sh_valid[lane] = isfinite(g) && g >= 0.0 && g < 1.0 && isfinite(zeta) &&
                       gl::set_valid(p.t0[s], p.period[s], p.a_rs[s], p.b[s], p.ecc[s],
                                     p.omega[s], p.k[s], p.f[s], p.eta[s], p.xi[s],
                                     p.u1[s], p.u2[s], p.exptime[s], ns);
    }
  }
  __syncthreads();
  if (!live || role != 0) return;
  const bool ok = orbit_ok && sh_valid[lane];
  sets[s].flags = ok ? (sh_win[lane] | sh_tay[lane]) : gl::kSetInvalid;
  if (!ok) atomicOr(status, kStatusInvalidSet);
  if (offsets) {
    bool bad = offsets[s] > offsets[s + 1] || (s == 0 && offsets[0] != 0) ||
               (s == n_sets - 1 && offsets[n_sets] != n_total);
    if (bad) atomicOr(status, kStatusBadOffsets);
  }
}

// index of the set owning exposure j in a CSR layout (offsets non-decreasing)
__device__ __forceinline__ int64_t owner_of(const int64_t* offsets, int64_t n_sets, int64_t j) {
  int64_t lo = 0, hi = n_sets;   // offsets[lo] <= j < offsets[hi]
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename R>
__global__ void __launch_bounds__(256) gl_curve_kernel(const SetConst* __restrict__ sets,
                                                       const double* __restrict__ t,
                                                       const int64_t* __restrict__ offsets,
                                                       int64_t n_times, int64_t n_sets,
                                                       int64_t n_total,
                                                       double* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_total;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t s;
    double tj;
    if (offsets) {
      s = owner_of(offsets, n_sets, j);
      tj = t[j];
    } else {
      s = j / n_times;
      tj = t[j - s * n_times];
    }
    const SetConst& c = sets[s];
    if (c.flags & gl::kSetInvalid) {
      out[j] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    double tau = gl::wrap_tau(c, tj);
    int ns = c.nsuper;
    if (!gl::exposure_in_window(c, tau)) {
      out[j] = 1.0;
      continue;
    }
    double acc = 0.0;
    for (int q = 0; q < ns; ++q) {
      double tq = tau + gl::subexposure_offset(q, ns, c.exptime);
      acc += gl::subexposure_flux<R>(c, tq, set_rule<R>(c, kRuleDefault));
    }
    out[j] = acc / ns;
  }
}

// max |a - b| over n doubles (NaN counts as infinite), into *err (non-negative
// doubles order like their bit patterns)
__global__ void gl_maxdiff_kernel(const double* a, const double* b, int64_t n,
                                  unsigned long long* err) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = fabs(a[i] - b[i]);
    if (!(d <= m)) m = isnan(d) ? INFINITY : d;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(err, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------------------ light-curve kernels
// Two ways to the same numbers (chosen by gl_item_pipeline):
//
// Item pipeline (default), four flat kernels after the per-set constants:
//   gl_win_kernel    two exposures per thread and pass: the conservative FP32
//                    window test (no FP64 instruction); exposures outside get
//                    flux 1, the rest are appended to a kept-exposure list
//   gl_expgeo_kernel one thread per kept exposure: the exact FP64 window test
//                    (exposures that fail it get flux 1) and the midpoint state
//                    (FP64 Kepler);
//                    then the block's threads together: the position and overlap
//                    class of each sub-exposure; items that meet the disk go to
//                    global queues (crossing items from the back of one, whole
//                    ellipses from its front, whole ellipses that may have two
//                    maxima of g to a second)
//   gl_items_quad_kernel   the quadrature of every queued item, warps spread over
//                    the whole GPU, crossing (heavier) items first
//   gl_items_sum_kernel    FP64 mean of each exposure, in sub-exposure order
// When the workspace is full, an exposure is finished by the thread that holds it.
//
// Tiles (gl_lc_kernel): one CTA takes tiles of TILE consecutive exposures from an
// atomic tile counter and finishes them itself:
//   phase 0  one thread per exposure: conservative FP32 window test; exposures
//            outside get flux 1 at once, the rest are compacted in shared memory
//   phase 1  one thread per kept exposure: exact FP64 window test (exposures that
//            fail it get flux 1 and no sub-exposure items) and, for the FP32C
//            path, the FP64 Kepler state at the exposure midpoint
//   rounds   up to CAP sub-exposure items at a time:
//            2: position (cubic Taylor step in FP32 from the midpoint state, or
//               FP64 Kepler per item), classification, queueing
//            3: whole-ellipse items (full-turn quadrature)
//            4: crossing items (roots, arcs)
//            5: FP64 accumulation of 1 - deficit per exposure, in item order
//   phase 6  mean over the exposure's sub-exposures -> out
//
// Every exposure's midpoint state, every item's geometry and deficit come from
// the same compiled functions (exposure_prep, item_geometry, item_deficit; the
// FP32 Taylor geometry, taylor_item, is written with fixed-rounding operations
// and gives the same bits inlined or not) and every exposure is summed in
// sub-exposure order, so the two ways, and any workspace size, give
// bit-identical results.
struct LcArgs {
  const SetConst* sets;
  const double* t;
  const int64_t* offsets;
  int64_t n_times, n_sets, n_total;
  double* out;
  unsigned int* tile_counter;
  unsigned long long* counts;   // instrumented instances: GL_COUNT_* slots
  int n_tiles, tile, cap;
  int rule_idx;                 // FP32 quadrature order: index into c_rule32_tuned, -1 = default
  // item pipeline workspace
  void* ipos;                   // R[3 * item_cap]: x0, y0, 1 - x0^2 - y0^2 of each item
  void* idef;                   // R[item_cap]: deficit (c0 I0 + c1 I1 + c2 I2) / F0 of each item
  int* iset;                    // parameter set of each item
  int* iq;                      // whole-ellipse items from the front, crossing items from the back
  int* ihq;                     // whole-ellipse items whose boundary may have two inner maxima
  int *rj, *rfirst, *rns;       // exposure records: output index, first item, sub-exposures
  int* klist;                   // kept exposures (output index); n_total entries
  int* kset;                    // their parameter sets; n_total entries
  unsigned long long* ictr;     // kIc* counters, then kSmspSlots 32-bit crossing-batch counters
  int n_smsp;                   // SM sub-partitions of the device (4 per SM)
  int64_t item_cap;
  int* ovlist;                  // kept-list indices of exposures left to the sum kernel
};

enum : int {
  kIcItems = 0, kIcRecs = 1, kIcFull = 2, kIcPart = 3, kIcFetch = 4, kIcKept = 5, kIcOver = 6,
  kIcFetchP = 7, kIcHeavy = 8, kIcFetchH = 9 /* (unused: heavy batches go by warp index) */,
  kIcSlots = 10,
  // per-sub-partition counters of crossing batches (32-bit, after the kIc slots)
  kSmspSlots = 1024,
  kIcWords = kIcSlots + kSmspSlots / 2   // 64-bit words zeroed by every step
};

// Index of the batch's FP32 quadrature order in c_rule32_tuned (-1 = default).
__device__ __forceinline__ int rule_base(int idx) { return idx < 0 ? kRuleDefault : idx; }

template <typename R>
struct LcSmem {
  // byte offsets into dynamic shared memory
  static __host__ __device__ size_t acc(int tile) { return 0; }
  static __host__ __device__ size_t tau(int tile) { return acc(tile) + 8 * (size_t)tile; }
  static __host__ __device__ size_t mid(int tile) { return tau(tile) + 8 * (size_t)tile; }
  static __host__ __device__ size_t ej(int tile) { return mid(tile) + sizeof(gl::MidState) * (size_t)tile; }
  static __host__ __device__ size_t es(int tile) { return ej(tile) + 4 * (size_t)tile; }
  static __host__ __device__ size_t ens(int tile) { return es(tile) + 4 * (size_t)tile; }
  static __host__ __device__ size_t ebase(int tile) { return ens(tile) + 4 * (size_t)tile; }
  static __host__ __device__ size_t eflag(int tile) { return ebase(tile) + 4 * (size_t)(tile + 1); }
  static __host__ __device__ size_t pos(int tile) { return (eflag(tile) + 4 * (size_t)tile + 15) & ~(size_t)15; }
  static __host__ __device__ size_t def(int tile, int cap) { return pos(tile) + 3 * sizeof(R) * (size_t)cap; }
  static __host__ __device__ size_t qf(int tile, int cap) { return def(tile, cap) + sizeof(R) * (size_t)cap; }
  static __host__ __device__ size_t qp(int tile, int cap) { return qf(tile, cap) + 4 * (size_t)cap; }
  static __host__ __device__ size_t total(int tile, int cap) { return qp(tile, cap) + 4 * (size_t)cap; }
};

enum : int { kExpDead = 1, kExpTaylor = 2 };

// exclusive prefix sum over the block of one int per thread; returns the
// prefix, writes the total to *total (all threads)
template <int NT>
__device__ __forceinline__ int block_scan(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < NT / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  int before = (w > 0 ? warp_tot[w - 1] : 0) + x - v;
  *total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return before;
}

// Warp-aggregated add to a device counter (instrumented instances only).
__device__ __forceinline__ void count_add(unsigned long long* c, bool pred) {
  unsigned m = __ballot_sync(__activemask(), pred);
  if (m && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(c, (unsigned long long)__popc(m));
}

// Exposure at time t: tau (t - t0 wrapped about the conjunction), the exact FP64
// window test (kExpDead outside) and, for the FP32C path of a set that allows
// it, the FP64 Kepler state at the midpoint for the cubic Taylor steps.
// exposure_prep, item_geometry and item_deficit are compiled once (not inlined),
// so every call site runs the same instructions: inlined copies may contract
// multiply-adds differently.
template <typename R>
__device__ __noinline__ int exposure_prep(const SetConst& c, double t, double* tau_out,
                                          gl::MidState* mid) {
  const double tau = gl::wrap_tau(c, t);
  *tau_out = tau;
  if (!gl::exposure_in_window(c, tau)) return kExpDead;
  if (sizeof(R) == 4 && (c.flags & gl::kSetTaylor)) {
    // with one sub-exposure it sits at the midpoint: no derivatives needed (the
    // Taylor step with dt = 0 returns the midpoint values unchanged)
    *mid = gl::mid_state_at(c, tau, c.nsuper != 1);
    return kExpTaylor;
  }
  return 0;
}

// Sky position (x0, y0, 1 - x0^2 - y0^2 in precision R) and overlap class of the
// sub-exposure at offset (twice / 2) * sub_step from the exposure midpoint tau:
// a cubic Taylor step in FP32 from the midpoint state when the set allows it,
// otherwise the FP64 Kepler solve.
template <typename R>
__device__ __noinline__ int item_geometry(const SetConst& c, int flag, const gl::MidState& mid,
                                          double tau, int twice, R* x, R* y, R* o) {
  if (flag & kExpTaylor) {
    float xf, yf, of;
    const int cls = gl::taylor_item(c, mid, twice, &xf, &yf, &of);
    *x = (R)xf;
    *y = (R)yf;
    *o = (R)of;
    return cls;
  }
  double xd, yd, zd;
  gl::sky_position(c, tau + 0.5 * (double)twice * c.sub_step, &xd, &yd, &zd);
  *x = (R)xd;
  *y = (R)yd;
  *o = (R)((1.0 - xd) * (1.0 + xd) - yd * yd);
  return gl::classify(c, xd, yd, zd);
}

// Deficit of a whole ellipse on the disk whose g has a single maximum (the common
// item; a small function of its own), in precision R.
template <typename R>
__device__ __noinline__ R whole_deficit(const SetConst& c, R x, R y, R o, int base) {
  R I[3];
  gl::whole_single_moments<R>(c, x, y, o, set_rule<R>(c, base), I);
  return (gl::pick<R>(c.c0, c.fc0) * I[0] + gl::pick<R>(c.c1, c.fc1) * I[1] +
          gl::pick<R>(c.c2, c.fc2) * I[2]) * gl::pick<R>(c.invF0, c.finvF0);
}

// Deficit of an item of class CLS (kPartial: the boundary may cross the limb;
// kFull: a whole ellipse whose g may have two maxima), each class compiled on its
// own so that each routine carries only its own branch of occulted_r.
template <typename R, int CLS>
__device__ __noinline__ R class_deficit(const SetConst& c, R x, R y, R o, int base) {
  R I[3];
  gl::occulted_r<R>(c, x, y, o, CLS, set_rule<R>(c, base), I);
  return (gl::pick<R>(c.c0, c.fc0) * I[0] + gl::pick<R>(c.c1, c.fc1) * I[1] +
          gl::pick<R>(c.c2, c.fc2) * I[2]) * gl::pick<R>(c.invF0, c.finvF0);
}

// Deficit of one item: limb-darkened occulted flux over F0, in precision R, by
// the routine of its kind (every path calls these same routines, so that they
// agree to the bit).
template <typename R>
__device__ __noinline__ R item_deficit(const SetConst& c, R x, R y, R o, int cls, int base) {
  if (cls == gl::kPartial) return class_deficit<R, gl::kPartial>(c, x, y, o, base);
  if (!gl::maybe_two_maxima(c, (float)x, (float)y)) return whole_deficit<R>(c, x, y, o, base);
  return class_deficit<R, gl::kFull>(c, x, y, o, base);
}

// Flux of one live exposure computed by the calling thread alone (the item
// pipeline's fallback when its workspace is full).
template <typename R>
__device__ double exposure_local(const SetConst& c, int flag, const gl::MidState& mid, double tau,
                                 int ns, int base) {
  double acc = 0.0;
  for (int q = 0; q < ns; ++q) {
    R x, y, o;
    const int cls = item_geometry<R>(c, flag, mid, tau, 2 * q + 1 - ns, &x, &y, &o);
    const R d = cls == gl::kOut ? R(0) : item_deficit<R>(c, x, y, o, cls, base);
    acc += gl::to_f64(d);
  }
  return exposure_mean(acc, ns);
}

template <typename R, int NT, bool COUNT>
__global__ void __launch_bounds__(NT) gl_lc_kernel(LcArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int warp_tot[32];
  __shared__ int s_tile, s_nf, s_np;
  __shared__ long long s_first;
  const int tile_sz = a.tile, cap = a.cap;
  double* e_acc = (double*)(smem + LcSmem<R>::acc(tile_sz));
  double* e_tau = (double*)(smem + LcSmem<R>::tau(tile_sz));
  gl::MidState* e_mid = (gl::MidState*)(smem + LcSmem<R>::mid(tile_sz));
  int* e_j = (int*)(smem + LcSmem<R>::ej(tile_sz));
  int* e_s = (int*)(smem + LcSmem<R>::es(tile_sz));
  int* e_ns = (int*)(smem + LcSmem<R>::ens(tile_sz));
  int* e_base = (int*)(smem + LcSmem<R>::ebase(tile_sz));
  int* e_flag = (int*)(smem + LcSmem<R>::eflag(tile_sz));
  R* it_pos = (R*)(smem + LcSmem<R>::pos(tile_sz));
  R* it_def = (R*)(smem + LcSmem<R>::def(tile_sz, cap));
  int* q_full = (int*)(smem + LcSmem<R>::qf(tile_sz, cap));
  int* q_part = (int*)(smem + LcSmem<R>::qp(tile_sz, cap));
  const int rb = rule_base(a.rule_idx);
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= a.n_tiles) break;
    const int64_t j0 = (int64_t)tile * tile_sz;
    if (a.offsets && tid == 0) s_first = owner_of(a.offsets, a.n_sets, j0);
    __syncthreads();

    // ---- phase 0: conservative window test, compaction
    int keep = 0, my_s = 0, my_ns = 0;
    double my_t = 0.0;
    int64_t j = j0 + tid;
    if (tid < tile_sz && j < a.n_total) {
      int64_t ti;   // index into t: CSR shares the exposure index, a shared grid repeats
      if (a.offsets) {
        int64_t s = s_first;
        while (s + 1 < a.n_sets && a.offsets[s + 1] <= j) ++s;
        my_s = (int)s;
        ti = j;
      } else {
        my_s = (int)((unsigned)j / (unsigned)a.n_times);
        ti = j - (int64_t)my_s * a.n_times;
      }
      const SetConst& c = a.sets[my_s];
      my_t = a.t[ti];
      if (c.flags & gl::kSetInvalid) {
        a.out[j] = __longlong_as_double(0x7ff8000000000000LL);
      } else if (gl::window_maybe(c, my_t)) {
        keep = 1;
        my_ns = c.nsuper;
      } else {
        a.out[j] = 1.0;
      }
    }
    if (COUNT) {
      count_add(&a.counts[GL_COUNT_EXPOSURES], tid < tile_sz && j < a.n_total);
      count_add(&a.counts[GL_COUNT_KEPT], keep != 0);
    }
    int m;
    int slot = block_scan<NT>(keep, warp_tot, &m);
    if (keep) {
      e_j[slot] = (int)j;
      e_s[slot] = my_s;
      e_ns[slot] = my_ns;
      e_tau[slot] = my_t;   // the time; phase 1 turns it into tau
    }
    __syncthreads();
    if (m == 0) continue;

    // ---- phase 1: exact window test and midpoint state
    for (int i = tid; i < m; i += NT) {
      const SetConst& c = a.sets[e_s[i]];
      double tau;
      const int fl = exposure_prep<R>(c, e_tau[i], &tau, &e_mid[i]);
      if (fl & kExpDead) {
        a.out[e_j[i]] = 1.0;
        e_ns[i] = 0;   // no sub-exposure items
      }
      e_tau[i] = tau;
      e_flag[i] = fl;
      e_acc[i] = 0.0;
      if (COUNT) {
        atomicAdd(&a.counts[GL_COUNT_IN_WINDOW], (unsigned long long)!(fl & kExpDead));
        atomicAdd(&a.counts[GL_COUNT_KEPLER], (unsigned long long)((fl & kExpTaylor) ? 1 : 0));
      }
    }
    __syncthreads();
    int M;
    int base = block_scan<NT>(tid < m ? e_ns[tid] : 0, warp_tot, &M);
    if (tid < m) e_base[tid] = base;
    if (tid == 0) e_base[m] = M;
    __syncthreads();

    for (int r0 = 0; r0 < M; r0 += cap) {
      const int nr = min(cap, M - r0);
      if (tid == 0) {
        s_nf = 0;
        s_np = 0;
      }
      __syncthreads();
      // ---- phase 2: positions and classes
      for (int k = tid; k < nr; k += NT) {
        int it = r0 + k;
        int lo = 0, hi = m;   // e_base[lo] <= it < e_base[hi]: skips empty ranges
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (e_base[mid] <= it) lo = mid; else hi = mid;
        }
        const int i = lo, q = it - e_base[i];
        it_def[k] = R(0);
        const SetConst& c = a.sets[e_s[i]];
        R x, y, o;
        const int cls = item_geometry<R>(c, e_flag[i], e_mid[i], e_tau[i], 2 * q + 1 - e_ns[i],
                                         &x, &y, &o);
        if (COUNT) {
          atomicAdd(&a.counts[GL_COUNT_ITEMS], 1ull);
          if (!(e_flag[i] & kExpTaylor)) atomicAdd(&a.counts[GL_COUNT_ITEM_KEPLER], 1ull);
          if (cls == gl::kFull) atomicAdd(&a.counts[GL_COUNT_FULL], 1ull);
          if (cls == gl::kPartial) atomicAdd(&a.counts[GL_COUNT_PARTIAL], 1ull);
        }
        if (cls == gl::kOut) continue;
        it_pos[3 * k] = x;
        it_pos[3 * k + 1] = y;
        it_pos[3 * k + 2] = o;
        int packed = k | (i << 16);
        if (cls == gl::kFull) q_full[atomicAdd(&s_nf, 1)] = packed;
        else q_part[atomicAdd(&s_np, 1)] = packed;
      }
      __syncthreads();
      // ---- phases 3 and 4: quadrature, whole-ellipse items first
      const int nf = s_nf, np = s_np;
      for (int u = tid; u < nf + np; u += NT) {
        int packed = u < nf ? q_full[u] : q_part[u - nf];
        int k = packed & 0xffff, i = packed >> 16;
        const SetConst& c = a.sets[e_s[i]];
        it_def[k] = item_deficit<R>(c, it_pos[3 * k], it_pos[3 * k + 1], it_pos[3 * k + 2],
                                    u < nf ? gl::kFull : gl::kPartial, rb);
      }
      __syncthreads();
      // ---- phase 5: FP64 accumulation in item order
      for (int i = tid; i < m; i += NT) {
        int b0 = max(e_base[i], r0), b1 = min(e_base[i + 1], r0 + nr);
        double acc = e_acc[i];
        for (int it = b0; it < b1; ++it) acc += gl::to_f64(it_def[it - r0]);
        e_acc[i] = acc;
      }
      __syncthreads();
    }
    // ---- phase 6: exposure means (exposures that failed the exact test are done)
    for (int i = tid; i < m; i += NT)
      if (e_ns[i] > 0) a.out[e_j[i]] = exposure_mean(e_acc[i], e_ns[i]);
    __syncthreads();
  }
}

// Item pipeline, stage 1: the conservative FP32 window test of every exposure.
// Each block walks a contiguous range in passes of 256 x U exposures; a thread
// first issues the loads of its U times (coalesced, none behind a store), then
// tests them.  It keeps the FP32 window constants of its current set in
// registers and the index where the next set starts; a pass in which every
// lane's exposures lie in the set it holds (almost all of them) takes a path
// with no lookup at all.  Exposures that pass are appended to the kept list;
// the exact FP64 test is the exposure kernel's (exposure_prep), so no FP64
// instruction runs here.
constexpr int kWinU = 2;

// start of set s + 1 relative to the range start lo (clamped to the int range)
__device__ __forceinline__ int next_set_start(const int64_t* offs, int64_t n_times,
                                              int64_t n_sets, int s, int64_t lo) {
  if (s + 1 >= n_sets) return INT_MAX;
  const int64_t b = (offs ? offs[s + 1] : (int64_t)(s + 1) * n_times) - lo;
  return b > (int64_t)INT_MAX ? INT_MAX : (int)b;
}

// window test of exposure lo + i of set s at time t: flux 1 (NaN for an invalid
// set) outside, else a kept-list entry (one atomic add per warp with keeps); all
// 32 lanes call it, lanes without an exposure with valid = false
__device__ __forceinline__ void win_one(const LcArgs& a, double* __restrict__ out,
                                        const gl::WinTest& w, int64_t lo, int i, int s,
                                        double t, bool valid) {
  const bool dead = w.flags & gl::kSetInvalid;
  const bool keep = valid && !dead && gl::window_maybe(w, t);
  if (valid && !keep) __stcs(out + i, dead ? __longlong_as_double(0x7ff8000000000000LL) : 1.0);
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (bal) {
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.ictr[kIcKept], (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) {   // at most n_total entries
      const long long slot = (long long)base + __popc(bal & ((1u << lane) - 1u));
      a.klist[slot] = (int)(lo + i);
      a.kset[slot] = s;
    }
  }
}

template <int U>
__global__ void __launch_bounds__(256) gl_win_kernel(LcArgs a) {
  __shared__ int s_first;
  pdl_wait();
  const int64_t per = (((a.n_total + gridDim.x - 1) / gridDim.x) + 31) & ~(int64_t)31;
  const int64_t lo = (int64_t)blockIdx.x * per;
  const int64_t hi = min(a.n_total, lo + per);
  if (lo >= hi) return;   // whole block
  const int n = (int)(hi - lo);   // n_total < 2^31
  const int tid = threadIdx.x;
  const double* __restrict__ tt = a.t;
  double* __restrict__ out = a.out + lo;
  const SetConst* __restrict__ sets = a.sets;
  const int64_t* __restrict__ offs = a.offsets;
  int s_run;   // owner of this thread's previous exposure
  if (offs) {
    if (tid == 0) s_first = (int)owner_of(offs, a.n_sets, lo);
    __syncthreads();
    s_run = s_first;
  } else {
    s_run = (int)((unsigned)(lo + tid) / (unsigned)a.n_times);
  }
  int nb = next_set_start(offs, a.n_times, a.n_sets, s_run, lo);
  int sc = -1;   // set whose constants wc holds
  gl::WinTest wc{};
  for (int i0 = 0; i0 < n; i0 += 256 * U) {
    const int il = i0 + (U - 1) * 256 + tid;   // this thread's last exposure of the pass
    double tv[U];
    if (__all_sync(0xffffffffu, il < n && il < nb && s_run == sc)) {
      // every exposure of the warp's pass exists and lies in the lane's cached set
      const double* tb = offs ? tt + lo : tt + (lo - (int64_t)s_run * a.n_times);
#pragma unroll
      for (int u = 0; u < U; ++u)
        tv[u] = offs ? __ldcs(tb + i0 + u * 256 + tid) : __ldg(tb + i0 + u * 256 + tid);
#pragma unroll
      for (int u = 0; u < U; ++u) win_one(a, out, wc, lo, i0 + u * 256 + tid, s_run, tv[u], true);
      continue;
    }
    int sv[U];
    if (offs) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * 256 + tid;
        tv[u] = i < n ? __ldcs(tt + lo + i) : 0.0;   // read once: do not keep in L2
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * 256 + tid;
        if (i < n)
          while (i >= nb) nb = next_set_start(offs, a.n_times, a.n_sets, ++s_run, lo);
        sv[u] = s_run;
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * 256 + tid;
        tv[u] = 0.0;
        if (i < n) {
          while (i >= nb) nb = next_set_start(offs, a.n_times, a.n_sets, ++s_run, lo);
          tv[u] = __ldg(tt + (lo + i - (int64_t)s_run * a.n_times));
        }
        sv[u] = s_run;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * 256 + tid;
      if (i < n && sv[u] != sc) {
        sc = sv[u];
        wc = gl::win_test(sets[sc]);
      }
      win_one(a, out, wc, lo, i, sv[u], tv[u], i < n);
    }
  }
}

// Item pipeline, stage 2 (kept exposures and their sub-exposures in one kernel):
// the first NE threads of a block take one kept exposure each: exact
// window and FP64 midpoint state, kept in shared memory, with one atomic add each
// reserving the block's item slots and records.  Then all threads expand the
// NE exposures' sub-exposures, four per thread and pass (item i
// belongs to the exposure whose slot range holds i, found by binary search over
// the block's offsets): FP32 Taylor position and overlap class (taylor_item, the
// same fixed-rounding code as everywhere else, inlined so that a thread's four
// items overlap), queued with one atomic add per pass and queue.  Exposures that
// do not fit the workspace go to the overflow list.
// NT = 64: every thread also takes an exposure (the most FP64 warps per SM, for
// large batches); NT = 256: 32 exposures per block iteration, expanded by eight
// times the threads (shorter per-thread chains and twice the blocks with work,
// for small batches; 64 or 16 per block measured slower there).  The autotuner
// chooses.
constexpr int kFuseExp = 64;

template <typename R, int NT>
__global__ void __launch_bounds__(NT) gl_expgeo_kernel(LcArgs a) {
  constexpr int NE = NT == 256 ? kFuseExp / 2 : kFuseExp, V = 4;
  __shared__ int warp_tot[32];
  __shared__ long long s_base, s_rec, s_q[3];
  __shared__ int s_fits, s_total, s_n[3];
  __shared__ int s_off[NE], s_st[NE], s_fl[NE], s_ns[NE];
  __shared__ double s_tau[NE];
  __shared__ gl::MidState s_mid[NE];
  pdl_wait();
  const int tid = threadIdx.x;
  // the block's first kept-list entries are loaded together with the kept count
  // (one dependent round trip less; an entry past the count is never used)
  const long long kf = (long long)blockIdx.x * NE + tid;
  int jf = 0, sf = 0;
  if (tid < NE && kf < a.n_total) {
    jf = a.klist[kf];
    sf = a.kset[kf];
  }
  const long long nk = (long long)a.ictr[kIcKept];
  R* ipos = (R*)a.ipos;
  R* idef = (R*)a.idef;
  for (long long k0 = (long long)blockIdx.x * NE; k0 < nk; k0 += (long long)gridDim.x * NE) {
    const long long k = k0 + tid;
    int j = 0, st = 0, fl = kExpDead, ns = 0;
    double tau = 0.0;
    gl::MidState mid;
    if (tid < NE && k < nk) {
      j = k == kf ? jf : a.klist[k];
      st = k == kf ? sf : a.kset[k];
      const int64_t ti = a.offsets ? (int64_t)j : (int64_t)j - (int64_t)st * a.n_times;
      fl = exposure_prep<R>(a.sets[st], a.t[ti], &tau, &mid);
      if (fl & kExpDead) a.out[j] = 1.0;
      else ns = a.sets[st].nsuper;
    }
    int total, n_live;
    const int off = block_scan<NT>(ns, warp_tot, &total);
    const int roff = block_scan<NT>(ns > 0 ? 1 : 0, warp_tot, &n_live);
    if (tid == 0) {
      long long b = 0, r = 0;
      int fits = 0;
      if (total > 0) {
        b = (long long)atomicAdd(&a.ictr[kIcItems], (unsigned long long)total);
        fits = b + total <= a.item_cap;
        if (fits) r = (long long)atomicAdd(&a.ictr[kIcRecs], (unsigned long long)n_live);
      }
      s_base = b;
      s_rec = r;
      s_fits = fits;
      s_total = total;
      s_n[0] = s_n[1] = s_n[2] = 0;
    }
    if (tid < NE) {
      s_off[tid] = off;
      s_st[tid] = st;
      s_fl[tid] = fl;
      s_ns[tid] = ns;
      s_tau[tid] = tau;
      s_mid[tid] = mid;
    }
    __syncthreads();
    if (ns > 0) {
      if (s_fits) {
        const long long r = s_rec + roff;
        a.rj[r] = j;
        a.rfirst[r] = (int)(s_base + off);
        a.rns[r] = ns;
      } else {
        a.ovlist[atomicAdd(&a.ictr[kIcOver], 1ull)] = (int)k;
      }
    }
    if (s_fits) {
      const int tot = s_total;
      for (int i0 = 0; i0 < tot; i0 += V * NT) {
        int qk[V], slot[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int i = i0 + tid + v * NT;
          qk[v] = -1;
          slot[v] = 0;
          if (i < tot) {
            int lo = 0, hi = NE;   // largest e with s_off[e] <= i (it has items)
            while (hi - lo > 1) {
              const int md = (lo + hi) >> 1;
              if (s_off[md] <= i) lo = md;
              else hi = md;
            }
            const int e = lo, q = i - s_off[lo];
            const SetConst& c = a.sets[s_st[e]];
            const long long g = s_base + i;
            R x, y, o;
            int cls;
            if (s_fl[e] & kExpTaylor) {
              float xf, yf, of;
              cls = gl::taylor_item(c, s_mid[e], 2 * q + 1 - s_ns[e], &xf, &yf, &of);
              x = (R)xf;
              y = (R)yf;
              o = (R)of;
            } else {
              cls = item_geometry<R>(c, s_fl[e], s_mid[e], s_tau[e], 2 * q + 1 - s_ns[e], &x, &y,
                                     &o);
            }
            if (cls == gl::kOut) {
              idef[g] = R(0);
            } else {
              ipos[3 * g] = x;
              ipos[3 * g + 1] = y;
              ipos[3 * g + 2] = o;
              a.iset[g] = s_st[e];
              qk[v] = cls == gl::kPartial ? 1
                                          : (gl::maybe_two_maxima(c, (float)x, (float)y) ? 2 : 0);
              slot[v] = atomicAdd(&s_n[qk[v]], 1);
            }
          }
        }
        __syncthreads();
        if (tid < 3) {
          const int ic = tid == 0 ? kIcFull : (tid == 1 ? kIcPart : kIcHeavy);
          s_q[tid] = s_n[tid] ? (long long)atomicAdd(&a.ictr[ic], (unsigned long long)s_n[tid]) : 0;
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int g = (int)(s_base + i0 + tid + v * NT);
          if (qk[v] == 0) a.iq[s_q[0] + slot[v]] = g;
          else if (qk[v] == 1) a.iq[a.item_cap - 1 - (s_q[1] + slot[v])] = g;
          else if (qk[v] == 2) a.ihq[s_q[2] + slot[v]] = g;
        }
        __syncthreads();
        if (tid < 3) s_n[tid] = 0;
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// Item pipeline, stage 3: the quadrature of every queued item, spread over the
// whole GPU.  Each warp takes 32 consecutive queue positions at a time: crossing
// items (the heavier ones) first, then whole-ellipse items, so a warp's lanes
// mostly follow the same path and the last warps to finish have light work.
// SM index and warp slot of the calling warp (scheduling hints only: both may
// change under preemption, and nothing depends on them for correctness).
__device__ __forceinline__ unsigned smid_() {
  unsigned v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}
__device__ __forceinline__ unsigned warpid_() {
  unsigned v;
  asm volatile("mov.u32 %0, %%warpid;" : "=r"(v));
  return v;
}

// MINB = 4 allows 128 registers (4 resident CTAs per SM: the shortest warps,
// for batches with few items per sub-partition); MINB = 8 caps them at 64
// (8 CTAs per SM: more warps to hide latency, for large batches).  The
// autotuner chooses between the two.
template <typename R, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) gl_items_quad_kernel(LcArgs a) {
  pdl_wait();
  const int rb = rule_base(a.rule_idx);
  const long long np = (long long)a.ictr[kIcPart], nf = (long long)a.ictr[kIcFull];
  const long long nh = (long long)a.ictr[kIcHeavy];
  const R* ipos = (const R*)a.ipos;
  R* idef = (R*)a.idef;
  const int lane = threadIdx.x & 31;
  auto run_item = [&](long long g, int cls) {
    const SetConst& c = a.sets[a.iset[g]];
    idef[g] = item_deficit<R>(c, ipos[3 * g], ipos[3 * g + 1], ipos[3 * g + 2], cls, rb);
  };
  auto run = [&](long long u, bool part) {
    if (part) {   // the back of the queue: items whose boundary may cross the limb
      const long long g = a.iq[a.item_cap - 1 - u];
      const SetConst& c = a.sets[a.iset[g]];
      idef[g] = class_deficit<R, gl::kPartial>(c, ipos[3 * g], ipos[3 * g + 1], ipos[3 * g + 2],
                                               rb);
    } else {   // the front of the queue: whole ellipses with a single maximum of g
      const long long g = a.iq[u];
      const SetConst& c = a.sets[a.iset[g]];
      idef[g] = whole_deficit<R>(c, ipos[3 * g], ipos[3 * g + 1], ipos[3 * g + 2], rb);
    }
  };
  // Pass 1, crossing items: a warp of them issues ~200 FP64 instructions and each
  // holds its sub-partition's FP64 unit ~64 cycles whatever the active lanes, so
  // their batches are spread evenly: at most `cap` per sub-partition, counted
  // per (SM, warp slot mod 4).  The counters only steer the spread; every batch
  // is still taken exactly once through the kIcFetchP counter.
  const long long pb = (np + 31) / 32;
  const unsigned cap = (unsigned)((pb + a.n_smsp - 1) / a.n_smsp);
  unsigned* smsp_ctr = (unsigned*)(a.ictr + kIcSlots);
  const unsigned key = (smid_() * 4u + (warpid_() & 3u)) & (kSmspSlots - 1);
  for (;;) {
    unsigned long long b = (unsigned long long)np;
    if (lane == 0 && atomicAdd(&smsp_ctr[key], 1u) < cap) b = atomicAdd(&a.ictr[kIcFetchP], 32ull);
    b = __shfl_sync(0xffffffffu, b, 0);
    if ((long long)b >= np) break;
    if ((long long)b + lane < np) run((long long)b + lane, true);
  }
  // Pass 2, whole-ellipse items that may have two inner maxima (their f_lin
  // takes two mapped arcs instead of one table rule: ~3x the work), then the
  // others, taken as they come, so that no heavy batch starts late.  The heavy
  // batches are few: they go to the warps by global warp index, counted from the
  // last warp (the last to reach the crossing counters), with no claim on a
  // shared counter (thousands of warps claiming at once queue on its address).
  {
    const long long hb = (nh + 31) / 32;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (long long bb = nw - 1 - gw; bb < hb; bb += nw) {
      const long long b = bb * 32;
      if (b + lane < nh) run_item(a.ihq[b + lane], gl::kFull);
    }
  }
  for (;;) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(&a.ictr[kIcFetch], 32ull);
    b = __shfl_sync(0xffffffffu, b, 0);
    if ((long long)b >= nf) break;
    if ((long long)b + lane < nf) run((long long)b + lane, false);
  }
  // Pass 3, crossing batches that pass 1 left (none unless warps met fewer
  // sub-partitions than the device has).
  for (;;) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(&a.ictr[kIcFetchP], 32ull);
    b = __shfl_sync(0xffffffffu, b, 0);
    if ((long long)b >= np) break;
    if ((long long)b + lane < np) run((long long)b + lane, true);
  }
}

// Item pipeline, stage 4: the FP64 mean of each exposure with items on the disk,
// summed in sub-exposure order (the deficits loaded eight at a time ahead of the
// adds, and widened to FP64 by integer operations: on B300 a conversion
// instruction holds the FP64 unit like an FP64 add).
// Exposures that did not fit the workspace are finished here, each by one
// thread (exact window, midpoint state, every sub-exposure in order).
// An exposure the workspace could not hold, finished by the calling thread
// (compiled apart from the sum kernel's loop, which it would otherwise swell).
template <typename R>
__device__ __noinline__ void finish_overflow(const LcArgs& a, int k, int rb) {
  const int j = a.klist[k], st = a.kset[k];
  const SetConst& c = a.sets[st];
  const int64_t ti = a.offsets ? (int64_t)j : (int64_t)j - (int64_t)st * a.n_times;
  double tau;
  gl::MidState mid;
  const int fl = exposure_prep<R>(c, a.t[ti], &tau, &mid);
  a.out[j] = (fl & kExpDead) ? 1.0 : exposure_local<R>(c, fl, mid, tau, c.nsuper, rb);
}

// Compiled for 8 resident blocks (32 registers): the sum loop needs few, and the
// fallback's call into the quadrature routines, which would raise the count to
// 128 (2 blocks per SM), spills instead; with 8 blocks per SM the uneven batch's
// step went from 580 to 551 us (MCMC batch unchanged).
template <typename R>
__global__ void __launch_bounds__(256, 8) gl_items_sum_kernel(LcArgs a) {
  pdl_wait();
  // the thread's first record is loaded together with the counters (one round
  // trip less; a slot past the records holds a value that is never used)
  const long long r0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int ns0 = 0, f0 = 0, j0 = 0;
  if (r0 < a.item_cap) {
    ns0 = a.rns[r0];
    f0 = a.rfirst[r0];
    j0 = a.rj[r0];
  }
  const long long nrec = (long long)a.ictr[kIcRecs];
  const long long nover = (long long)a.ictr[kIcOver];
  const R* idef = (const R*)a.idef;
  const int rb = rule_base(a.rule_idx);
  for (long long r = r0; r < nrec + nover; r += (long long)gridDim.x * blockDim.x) {
    if (r < nrec) {
      const bool first = r == r0;
      const int ns = first ? ns0 : a.rns[r];
      const R* d = idef + (first ? f0 : a.rfirst[r]);
      double acc = 0.0;
      for (int q0 = 0; q0 < ns; q0 += 8) {
        R v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = q0 + k < ns ? d[q0 + k] : R(0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (q0 + k < ns) acc += gl::to_f64(v[k]);
      }
      a.out[first ? j0 : a.rj[r]] = exposure_mean(acc, ns);
    } else {
      finish_overflow<R>(a, a.ovlist[r - nrec], rb);
    }
  }
}

// Tidally locked bodies (Appendix B): the projection follows the orbital angle,
// so every sub-exposure has its own ellipse.  One thread per exposure: window
// test, then per sub-exposure the FP64 Kepler position, the orbital angle alpha
// from conjunction (r cos alpha = x0 cos i - z sin i, r sin alpha = y0, the
// Keplerian reading of the paper's alpha), the locked projection and the same
// quadrature as the other paths; FP64 exposure mean in sub-exposure order.
template <typename R>
__global__ void __launch_bounds__(128) gl_locked_kernel(const SetConst* __restrict__ sets,
                                                        const double* __restrict__ t,
                                                        const int64_t* __restrict__ offsets,
                                                        int64_t n_times, int64_t n_sets,
                                                        int64_t n_total, int rule_idx,
                                                        double* __restrict__ out) {
  const int rb = rule_base(rule_idx);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_total;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t s;
    double tj;
    if (offsets) {
      s = owner_of(offsets, n_sets, j);
      tj = t[j];
    } else {
      s = j / n_times;
      tj = t[j - s * n_times];
    }
    const SetConst& c = sets[s];
    if (c.flags & gl::kSetInvalid) {
      out[j] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    const double tau = gl::wrap_tau(c, tj);
    const int ns = c.nsuper;
    if (!gl::exposure_in_window(c, tau)) {
      out[j] = 1.0;
      continue;
    }
    double acc = 0.0;
    for (int q = 0; q < ns; ++q) {
      double x0, y0, z;
      gl::sky_position(c, tau + gl::subexposure_offset(q, ns, c.exptime), &x0, &y0, &z);
      const int cls = gl::classify(c, x0, y0, z);   // R_eq bounds every projection
      if (cls == gl::kOut) {
        acc += 1.0;
        continue;
      }
      double ca = x0 * c.cosi - z * c.sini, sa = y0;
      const double ir = gl::rcp64(sqrt(ca * ca + sa * sa));
      SetConst cl;
      gl::locked_shape(c, ca * ir, sa * ir, &cl);
      const R d = item_deficit<R>(cl, (R)x0, (R)y0, (R)((1.0 - x0) * (1.0 + x0) - y0 * y0),
                                  cls, rb);
      acc += 1.0 - (double)d;
    }
    out[j] = acc / ns;
  }
}

// Spherical planet: one item per thread.
struct SpherePtrs {
  const double *x0, *y0, *z, *p, *u1, *u2;
};

template <typename R>
__global__ void __launch_bounds__(256) gl_sphere_kernel(SpherePtrs a, int64_t n, double* out,
                                                        int* status) {
  const NodeRule<R>& rl = rule<R>();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x0 = a.x0[i], y0 = a.y0[i], zz = a.z[i], p = a.p[i], u1 = a.u1[i], u2 = a.u2[i];
    double F0 = gl::kPi * (1.0 - u1 * (1.0 / 3.0) - u2 * (1.0 / 6.0));
    if (!(isfinite(x0) && isfinite(y0) && isfinite(zz) && isfinite(p) && p > 0.0 &&
          isfinite(u1) && isfinite(u2) && F0 > 0.0)) {
      out[i] = __longlong_as_double(0x7ff8000000000000LL);
      atomicOr(status, kStatusInvalidSet);
      continue;
    }
    double rho = sqrt(x0 * x0 + y0 * y0);
    if (zz > 0.0 || rho >= 1.0 + p) {
      out[i] = 1.0;
      continue;
    }
    R I[3];
    gl::sphere_moments<R>((R)rho, (R)p, (R)((1.0 - x0) * (1.0 + x0) - y0 * y0), rl, I);
    double def = (1.0 - u1 - 2.0 * u2) * (double)I[0] + (u1 + 2.0 * u2) * (double)I[1] +
                 u2 * (double)I[2];
    out[i] = 1.0 - def / F0;
  }
}

// ------------------------------------------------------------------ surrogate path
// Collect kernel: the exposure window, exact window and sub-exposure geometry of
// the FP32C light-curve kernel, but instead of integrating it writes every
// sub-exposure of an in-window exposure to global item arrays (position, 1 - r^2,
// set, class) and one record per exposure (output index, nsuper, first item).
// Items of an exposure are contiguous.  Exposures outside the window get flux 1
// at once.  One CTA per tile of exposures (atomic tile counter).
struct CollectArgs {
  const SetConst* sets;
  const double* t;
  const int64_t* offsets;
  int64_t n_times, n_sets, n_total;
  double* out;
  unsigned int* tile_counter;
  int n_tiles, tile;
  float *ix, *iy, *io;      // item geometry
  int *iset, *icls;         // item set and class (gl::kOut / kFull / kPartial)
  int64_t item_cap;
  unsigned long long* n_items;
  int *rj, *rns, *rfirst;   // exposure records
  int64_t rec_cap;
  unsigned long long* n_recs;
  int* status;
};

template <int NT>
__global__ void __launch_bounds__(NT) gl_collect_kernel(CollectArgs a) {
  __shared__ int warp_tot[32];
  __shared__ int s_tile;
  __shared__ long long s_first, s_item_base, s_rec_base;
  __shared__ int e_j[NT], e_s[NT], e_ns[NT], e_base[NT + 1], e_flag[NT];
  __shared__ double e_tau[NT];
  __shared__ gl::MidState e_mid[NT];
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= a.n_tiles) break;
    const int64_t j0 = (int64_t)tile * a.tile;
    if (a.offsets && tid == 0) s_first = owner_of(a.offsets, a.n_sets, j0);
    __syncthreads();
    int keep = 0, my_s = 0, my_ns = 0;
    double my_t = 0.0;
    int64_t j = j0 + tid;
    if (tid < a.tile && j < a.n_total) {
      int64_t ti;
      if (a.offsets) {
        int64_t s = s_first;
        while (s + 1 < a.n_sets && a.offsets[s + 1] <= j) ++s;
        my_s = (int)s;
        ti = j;
      } else {
        my_s = (int)((unsigned)j / (unsigned)a.n_times);
        ti = j - (int64_t)my_s * a.n_times;
      }
      const SetConst& c = a.sets[my_s];
      my_t = a.t[ti];
      if (c.flags & gl::kSetInvalid) {
        a.out[j] = __longlong_as_double(0x7ff8000000000000LL);
      } else if (gl::window_maybe(c, my_t)) {
        double tau = gl::wrap_tau(c, my_t);
        if (gl::exposure_in_window(c, tau)) {
          keep = 1;
          my_ns = c.nsuper;
          my_t = tau;
        } else {
          a.out[j] = 1.0;
        }
      } else {
        a.out[j] = 1.0;
      }
    }
    int m;
    int slot = block_scan<NT>(keep, warp_tot, &m);
    if (keep) {
      e_j[slot] = (int)j;
      e_s[slot] = my_s;
      e_ns[slot] = my_ns;
      e_tau[slot] = my_t;
    }
    __syncthreads();
    if (m == 0) continue;
    int M;
    int base = block_scan<NT>(tid < m ? e_ns[tid] : 0, warp_tot, &M);
    if (tid < m) e_base[tid] = base;
    if (tid == 0) {
      e_base[m] = M;
      s_item_base = (long long)atomicAdd(a.n_items, (unsigned long long)M);
      s_rec_base = (long long)atomicAdd(a.n_recs, (unsigned long long)m);
    }
    for (int i = tid; i < m; i += NT) {
      const SetConst& c = a.sets[e_s[i]];
      int fl = 0;
      if (c.flags & gl::kSetTaylor) {
        e_mid[i] = gl::mid_state_at(c, e_tau[i], true);
        fl = kExpTaylor;
      }
      e_flag[i] = fl;
    }
    __syncthreads();
    const long long ib = s_item_base, rb = s_rec_base;
    if (ib + M > a.item_cap || rb + m > a.rec_cap) {
      if (tid == 0) atomicOr(a.status, kStatusOverflow);
      for (int i = tid; i < m; i += NT) a.out[e_j[i]] = __longlong_as_double(0x7ff8000000000000LL);
      __syncthreads();
      continue;
    }
    for (int it = tid; it < M; it += NT) {
      int lo = 0, hi = m;
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (e_base[mid] <= it) lo = mid; else hi = mid;
      }
      const int i = lo, q = it - e_base[i];
      const SetConst& c = a.sets[e_s[i]];
      const int twice = 2 * q + 1 - e_ns[i];
      float x, y, o;
      int cls;
      if (e_flag[i] & kExpTaylor) {
        float zf;
        gl::taylor_position(e_mid[i], 0.5f * (float)twice * c.fsub_step, &x, &y, &zf, &o);
        cls = gl::classify_t<float>(c.freq, x, y, zf, 1e-6f);
      } else {
        double xd, yd, zd;
        gl::sky_position(c, e_tau[i] + 0.5 * (double)twice * c.sub_step, &xd, &yd, &zd);
        cls = gl::classify(c, xd, yd, zd);
        x = (float)xd;
        y = (float)yd;
        o = (float)((1.0 - xd) * (1.0 + xd) - yd * yd);
      }
      a.ix[ib + it] = x;
      a.iy[ib + it] = y;
      a.io[ib + it] = o;
      a.iset[ib + it] = e_s[i];
      a.icls[ib + it] = cls;
    }
    for (int i = tid; i < m; i += NT) {
      a.rj[rb + i] = e_j[i];
      a.rns[rb + i] = e_ns[i];
      a.rfirst[rb + i] = (int)(ib + e_base[i]);
    }
    __syncthreads();
  }
}

// Surrogate inputs of one item: seven features scaled to about [-1, 1]
//   rho = |centre|, psi = angle between the projected spin axis and the radial
//   direction folded into [0, pi/2] (the flux is unchanged by a half turn of the
//   ellipse and by reflection about the radial line), k, f, cos(eta), and the
//   Kipping coordinates q1 = (u1 + u2)^2, q2 = u1 / (2 (u1 + u2));
// and the equal-area sphere radius R_area = sqrt(dx dy2), scale = R_eq^2.
struct SurFeat {
  float f[7];
  float r_area, scale;
};
__device__ __forceinline__ SurFeat sur_features(double x0, double y0, double k, double f,
                                                double ce, double xi, double u1, double u2,
                                                double dx, double dy2, double req) {
  SurFeat o;
  double rho = sqrt(x0 * x0 + y0 * y0);
  double ang = -xi - atan2(y0, x0);
  double psi = ang - gl::kPi * floor(ang / gl::kPi);      // [0, pi)
  if (psi > 0.5 * gl::kPi) psi = gl::kPi - psi;           // [0, pi/2]
  double s = u1 + u2;
  double q1 = s * s, q2 = s > 0.0 ? u1 / (2.0 * s) : 0.0;
  o.f[0] = (float)(rho / 0.85 - 1.0);
  o.f[1] = (float)(psi * (4.0 / gl::kPi) - 1.0);
  o.f[2] = (float)((k - 0.105) / 0.095);
  o.f[3] = (float)((f - 0.45) / 0.45);
  o.f[4] = (float)(2.0 * ce - 1.0);
  o.f[5] = (float)(2.0 * q1 - 1.0);
  o.f[6] = (float)(2.0 * q2 - 1.0);
  o.r_area = (float)sqrt(dx * dy2);
  o.scale = (float)(req * req);
  return o;
}

constexpr int kSurBins = GL_SURROGATE_BINS;
__device__ __forceinline__ int sur_bin(int cls, double k) {
  int kb = (int)floor((k - 0.01) / (0.19 / 8.0));
  kb = kb < 0 ? 0 : (kb > 7 ? 7 : kb);
  return (cls == gl::kPartial ? 8 : 0) + kb;
}

// features, scale and the FP32 sphere deficit of every collected item
__global__ void gl_sur_features_kernel(const SetConst* __restrict__ sets, const ParamPtrs pp,
                                       const float* __restrict__ ix, const float* __restrict__ iy,
                                       const float* __restrict__ io, const int* __restrict__ iset,
                                       const int* __restrict__ icls,
                                       const unsigned long long* __restrict__ n_items,
                                       float* __restrict__ feat, float* __restrict__ scale,
                                       float* __restrict__ dsph) {
  const int64_t n = (int64_t)*n_items;
  const NodeRule<float>& rl = rule<float>();
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n;
       it += (int64_t)gridDim.x * blockDim.x) {
    if (icls[it] == gl::kOut) {
      for (int q = 0; q < 7; ++q) feat[it * 7 + q] = 0.f;
      scale[it] = 0.f;
      dsph[it] = 0.f;
      continue;
    }
    const int s = iset[it];
    const SetConst& c = sets[s];
    double x = ix[it], y = iy[it];
    SurFeat sf = sur_features(x, y, pp.k[s], pp.f[s], cos(pp.eta[s]), pp.xi[s], pp.u1[s], pp.u2[s],
                              c.dx, c.dy2, c.req);
    for (int q = 0; q < 7; ++q) feat[it * 7 + q] = sf.f[q];
    scale[it] = sf.scale;
    float I[3];
    float rho = sqrtf(ix[it] * ix[it] + iy[it] * iy[it]);
    gl::sphere_moments<float>(rho, sf.r_area, io[it], rl, I);   // io = 1 - rho^2
    dsph[it] = (c.fc0 * I[0] + c.fc1 * I[1] + c.fc2 * I[2]) * c.finvF0;
  }
}

// deficit = sphere deficit - predicted residual * scale; the items whose error
// bound (table[bin] * scale) exceeds the limit are queued for the exact path
__global__ void gl_sur_combine_kernel(const SetConst* __restrict__ sets,
                                      const double* __restrict__ kk, const int* __restrict__ iset,
                                      const int* __restrict__ icls,
                                      const unsigned long long* __restrict__ n_items,
                                      const float* __restrict__ that, const float* __restrict__ scale,
                                      const float* __restrict__ dsph, const float* __restrict__ table,
                                      float limit, float* __restrict__ def, int* __restrict__ fb,
                                      unsigned long long* __restrict__ n_fb) {
  const int64_t n = (int64_t)*n_items;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n;
       it += (int64_t)gridDim.x * blockDim.x) {
    int cls = icls[it];
    if (cls == gl::kOut) {
      def[it] = 0.f;
      continue;
    }
    float sc = scale[it];
    def[it] = dsph[it] - that[it] * sc;
    float bound = table[sur_bin(cls, kk[iset[it]])] * sc;
    if (!(bound <= limit)) fb[atomicAdd(n_fb, 1ull)] = (int)it;
  }
}

// exact FP32C deficit for the queued items
__global__ void gl_sur_fallback_kernel(const SetConst* __restrict__ sets, const float* __restrict__ ix,
                                       const float* __restrict__ iy, const float* __restrict__ io,
                                       const int* __restrict__ iset, const int* __restrict__ icls,
                                       const int* __restrict__ fb,
                                       const unsigned long long* __restrict__ n_fb,
                                       float* __restrict__ def) {
  const int64_t n = (int64_t)*n_fb;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int it = fb[u];
    const SetConst& c = sets[iset[it]];
    float I[3];
    gl::occulted_r<float>(c, ix[it], iy[it], io[it], icls[it], set_rule<float>(c, kRuleDefault), I);
    def[it] = (c.fc0 * I[0] + c.fc1 * I[1] + c.fc2 * I[2]) * c.finvF0;
  }
}

// exposure flux = mean over its sub-exposures of 1 - deficit (FP64, item order)
__global__ void gl_sur_reduce_kernel(const int* __restrict__ rj, const int* __restrict__ rns,
                                     const int* __restrict__ rfirst,
                                     const unsigned long long* __restrict__ n_recs,
                                     const float* __restrict__ def, double* __restrict__ out) {
  const int64_t n = (int64_t)*n_recs;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int f0 = rfirst[r], ns = rns[r];
    double acc = 0.0;
    for (int q = 0; q < ns; ++q) acc += 1.0 - (double)def[f0 + q];
    out[rj[r]] = acc / ns;
  }
}

// training data: features from sky positions and shapes
__global__ void gl_sur_geom_features_kernel(int64_t n, const double* x0, const double* y0,
                                            const double* k, const double* f, const double* eta,
                                            const double* xi, const double* u1, const double* u2,
                                            float* feat, float* scale, double* r_area, int* bin) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    SetConst c;
    gl::set_setup(0.0, 1.0, 10.0, 0.0, 0.0, 0.0, k[i], f[i], eta[i], xi[i], u1[i], u2[i], 0.0, 1, &c);
    SurFeat sf = sur_features(x0[i], y0[i], k[i], f[i], cos(eta[i]), xi[i], u1[i], u2[i], c.dx,
                              c.dy2, c.req);
    for (int q = 0; q < 7; ++q) feat[i * 7 + q] = sf.f[q];
    scale[i] = sf.scale;
    r_area[i] = sqrt(c.dx * c.dy2);
    int cls = gl::classify(c, x0[i], y0[i], -1.0);
    bin[i] = cls == gl::kOut ? -1 : sur_bin(cls, k[i]);
  }
}

// training targets: (F_oblate - F_sphere) / scale
__global__ void gl_sur_targets_kernel(int64_t n, const double* fo, const double* fs,
                                      const float* scale, float* t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    t[i] = scale[i] > 0.f ? (float)((fo[i] - fs[i]) / (double)scale[i]) : 0.f;
}

// log-likelihood per set: -chi^2 / 2 with chi^2 = sum_j ((flux_j - data_j) / sigma_j)^2
__global__ void gl_loglike_kernel(int64_t n_sets, int64_t n_times, const double* __restrict__ flux,
                                  const double* __restrict__ data, const double* __restrict__ sigma,
                                  double* __restrict__ ll) {
  int64_t s = blockIdx.x;
  if (s >= n_sets) return;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < n_times; j += blockDim.x) {
    double r = (flux[s * n_times + j] - data[j]) / sigma[j];
    acc += r * r;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ll[s] = -0.5 * red[0];
}

// ------------------------------------------------------------------ (mu, nu) and the ensemble
// Appendix A: mu = (f - 1)^2 + f (f - 2) cos(2 eta); f = f_min + (1 - f_min) nu with
// f_min = 1 - sqrt((mu + 1)/2); eta in [0, pi/2] from cos(2 eta) = (mu - (f-1)^2) /
// (f (f - 2)).  The printed nu(f, eta), joint density p(mu, nu) and the inverse
// transforms nu(u) = u^2 / (u^2 - 2u + 2), mu(w | nu).
__device__ __forceinline__ void munu_to_feta(double mu, double nu, double* f, double* eta) {
  const double fm = 1.0 - sqrt(0.5 * (mu + 1.0));
  const double ff = fm + (1.0 - fm) * nu;
  const double q = ff * (ff - 2.0);
  double c2 = q != 0.0 ? (mu - (ff - 1.0) * (ff - 1.0)) / q : 1.0;
  c2 = fmin(1.0, fmax(-1.0, c2));
  *f = ff;
  *eta = 0.5 * acos(c2);
}

__device__ __forceinline__ void feta_to_munu(double f, double eta, double* mu, double* nu) {
  const double c2 = cos(2.0 * eta), ce = cos(eta), q = f * (f - 2.0);
  *mu = (f - 1.0) * (f - 1.0) + q * c2;
  *nu = (2.0 + 2.0 * q * ce * ce + (f - 1.0) * sqrt(4.0 + 2.0 * q * (1.0 + c2))) /
        (2.0 + q * (1.0 + c2));
}

__device__ __forceinline__ void munu_prior_draw(double u, double w, double* mu, double* nu) {
  const double v = u * u / (u * u - 2.0 * u + 2.0);
  const double s = sqrt(v * (2.0 - v)), d = (v - 1.0) * (v - 1.0);
  *nu = v;
  *mu = (4.0 * w + 4.0 * (w * w - w) * s + 2.0 * (v * (v - 2.0) - 1.0) * w * w - d) / d;
}

__device__ __forceinline__ double log_p_munu(double mu, double nu) {
  const double x = nu * (nu - 2.0) * (mu * (nu - 1.0) * (nu - 1.0) + nu * (nu - 2.0) - 1.0);
  return x > 0.0 ? -1.5 * 0.69314718055994530942 - 0.5 * log(x) : -INFINITY;
}

enum : int { kMunuToFeta = 0, kFetaToMunu = 1, kMunuPrior = 2 };

__global__ void gl_munu_kernel(int op, int64_t n, const double* __restrict__ a,
                               const double* __restrict__ b, double* __restrict__ c,
                               double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x, y;
    if (op == kMunuToFeta) munu_to_feta(a[i], b[i], &x, &y);
    else if (op == kFetaToMunu) feta_to_munu(a[i], b[i], &x, &y);
    else munu_prior_draw(a[i], b[i], &x, &y);
    c[i] = x;
    d[i] = y;
  }
}

// Fit vector -> parameter sets (structure of arrays, 12 x m) and log prior:
// uniform inside [lo, hi] (also 0 <= q1, q2 <= 1, -1 <= mu <= 1, 0 <= nu <= 1),
// times p(mu, nu), which makes the prior on (f, eta) uniform in f and ~ cos(eta)
// (Appendix A); circular orbit (e = 0, w = pi/2); Kipping's map for (q1, q2).
// Rows outside the box get log prior -inf and a harmless valid parameter set.
__global__ void gl_ens_params_kernel(const double* __restrict__ x, int64_t m,
                                     const double* __restrict__ lo, const double* __restrict__ hi,
                                     double* __restrict__ soa, double* __restrict__ logprior) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[GL_FIT_DIM];
    bool in = true;
    for (int d = 0; d < GL_FIT_DIM; ++d) {
      v[d] = x[i * GL_FIT_DIM + d];
      in = in && v[d] >= lo[d] && v[d] <= hi[d];
    }
    const double mu = v[5], nu = v[6], q1 = v[8], q2 = v[9];
    // (mu = -1 or nu = 1 would give f = 1; b >= a_rs no inclination)
    in = in && mu > -1.0 && mu <= 1.0 && nu >= 0.0 && nu < 1.0 && q1 >= 0.0 && q1 <= 1.0 &&
         q2 >= 0.0 && q2 <= 1.0 && v[1] > 0.0 && v[2] > 1.0 && v[4] > 0.0 && v[3] >= 0.0 &&
         v[3] < v[2];
    double lp = in ? log_p_munu(mu, nu) : -INFINITY;
    if (!in) {   // any valid set: its light curve is not used
      for (int d = 0; d < GL_FIT_DIM; ++d) v[d] = 0.5 * (lo[d] + hi[d]);
      v[1] = fmax(v[1], 1.0);
      v[2] = fmax(v[2], 2.0);
      v[3] = 0.0;
      v[4] = 0.05;
      v[5] = 0.0;
      v[6] = 0.5;
      v[8] = 0.5;
      v[9] = 0.5;
    }
    double f, eta;
    munu_to_feta(v[5], v[6], &f, &eta);
    const double sq = sqrt(v[8]);
    double* o = soa;
    o[0 * m + i] = v[0];        // t0
    o[1 * m + i] = v[1];        // period
    o[2 * m + i] = v[2];        // a_rs
    o[3 * m + i] = v[3];        // b
    o[4 * m + i] = 0.0;         // ecc
    o[5 * m + i] = 0.5 * gl::kPi;   // omega
    o[6 * m + i] = v[4];        // k
    o[7 * m + i] = f;
    o[8 * m + i] = eta;
    o[9 * m + i] = v[7];        // xi
    o[10 * m + i] = 2.0 * sq * v[9];
    o[11 * m + i] = sq * (1.0 - 2.0 * v[9]);
    logprior[i] = lp;
  }
}

// Stretch-move proposals of one half (walkers k = 2 i + h) along lines through
// members of the other half: partner = 2 floor(r_j m) + (1 - h), z = ((a - 1) r_z + 1)^2 / a.
__global__ void gl_ens_propose_kernel(const double* __restrict__ walkers, int64_t m, int h,
                                      const double* __restrict__ rz, const double* __restrict__ rj,
                                      double a, double* __restrict__ prop, double* __restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = 2 * i + h;
    int64_t pj = (int64_t)(rj[i] * (double)m);
    if (pj >= m) pj = m - 1;
    if (pj < 0) pj = 0;
    const int64_t j = 2 * pj + (1 - h);
    const double zz = ((a - 1.0) * rz[i] + 1.0) * ((a - 1.0) * rz[i] + 1.0) / a;
    z[i] = zz;
    for (int d = 0; d < GL_FIT_DIM; ++d) {
      const double xj = walkers[j * GL_FIT_DIM + d];
      prop[i * GL_FIT_DIM + d] = xj + zz * (walkers[k * GL_FIT_DIM + d] - xj);
    }
  }
}

__global__ void gl_fill_kernel(double* __restrict__ x, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// log posterior = log prior + log likelihood (-inf outside the prior).
__global__ void gl_ens_post_kernel(int64_t m, const double* __restrict__ logprior,
                                   const double* __restrict__ ll, double* __restrict__ logpost) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    logpost[i] = isfinite(logprior[i]) ? logprior[i] + ll[i] : -INFINITY;
}

// Accept or reject the half's proposals with probability min(1, z^(D-1) p(Y)/p(X))
// (Goodman and Weare 2010), the zero-density cases written out so that no NaN
// decides a move: a proposal outside the prior (lp(Y) = -inf, or NaN) is never
// taken; a walker outside the prior (lp(X) = -inf) takes any proposal inside it;
// otherwise log(r_u) < (D - 1) log z + lp(Y) - lp(X).
__global__ void gl_ens_accept_kernel(double* __restrict__ walkers, double* __restrict__ logpost,
                                     int64_t m, int h, const double* __restrict__ prop,
                                     const double* __restrict__ z,
                                     const double* __restrict__ lp_new,
                                     const double* __restrict__ ru,
                                     unsigned long long* __restrict__ accepted) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = 2 * i + h;
    const double ly = lp_new[i], lx = logpost[k];
    bool take;
    if (!(ly > -INFINITY)) take = false;
    else if (!(lx > -INFINITY)) take = true;
    else take = log(ru[i]) < (GL_FIT_DIM - 1) * log(z[i]) + ly - lx;
    if (take) {
      for (int d = 0; d < GL_FIT_DIM; ++d) walkers[k * GL_FIT_DIM + d] = prop[i * GL_FIT_DIM + d];
      logpost[k] = lp_new[i];
      if (accepted) atomicAdd(accepted, 1ull);
    }
  }
}

struct SkyPtrs {
  const double *x0, *y0, *z, *k, *f, *eta, *xi, *u1, *u2;
};

template <typename R>
__global__ void __launch_bounds__(256) gl_sky_kernel(SkyPtrs p, int64_t n, double* out,
                                                     int* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    SetConst c;
    // orbit fields are placeholders: only the shape and LD parts are used
    bool ok = gl::set_setup(0.0, 1.0, 10.0, 0.0, 0.0, 0.0, p.k[i], p.f[i], p.eta[i], p.xi[i],
                            p.u1[i], p.u2[i], 0.0, 1, &c);
    double x0 = p.x0[i], y0 = p.y0[i], z = p.z[i];
    if (!ok || !isfinite(x0) || !isfinite(y0) || !isfinite(z)) {
      out[i] = __longlong_as_double(0x7ff8000000000000LL);
      atomicOr(status, kStatusInvalidSet);
      continue;
    }
    int cls = gl::classify(c, x0, y0, z);
    if (cls == gl::kOut) {
      out[i] = 1.0;
      continue;
    }
    R I[3];
    gl::occulted<R>(c, x0, y0, cls, set_rule<R>(c, kRuleDefault), I);
    R def = (R)c.c0 * I[0] + (R)c.c1 * I[1] + (R)c.c2 * I[2];
    out[i] = 1.0 - (double)def * c.invF0;
  }
}

// ------------------------------------------------------------------ the paper's scheme
// Geometry-level flux by the paper's own integration (Sec. 2): composite Simpson's
// rule over n_int uniform intervals of the ellipse angle th in [0, 2 pi) (periodic,
// so the end node weighs 2 like every even node), the boundary snapped to the
// limb where it lies outside the disk, no crossings.  One warp per evaluation:
// lanes take nodes j = lane, lane + 32, ..., each keeping a compensated sum in
// precision R; the lanes' sums are combined in FP64.  Positions with the planet
// behind the star or beyond rho >= 1 + R_eq give flux exactly 1.
template <typename R>
__global__ void __launch_bounds__(256) gl_simpson_kernel(SkyPtrs p, int64_t n, int n_int,
                                                         double* out, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarp) {
    SetConst c;
    const bool ok = gl::set_setup(0.0, 1.0, 10.0, 0.0, 0.0, 0.0, p.k[i], p.f[i], p.eta[i],
                                  p.xi[i], p.u1[i], p.u2[i], 0.0, 1, &c);
    const double x0 = p.x0[i], y0 = p.y0[i], z = p.z[i];
    if (!ok || !isfinite(x0) || !isfinite(y0) || !isfinite(z)) {
      if (lane == 0) {
        out[i] = __longlong_as_double(0x7ff8000000000000LL);
        atomicOr(status, kStatusInvalidSet);
      }
      continue;
    }
    if (gl::classify(c, x0, y0, z) == gl::kOut) {
      if (lane == 0) out[i] = 1.0;
      continue;
    }
    const R rx = (R)x0, ry = (R)y0, dx = gl::pick<R>(c.dx, c.fdx), dy1 = gl::pick<R>(c.dy1, c.fdy1),
            dy2 = gl::pick<R>(c.dy2, c.fdy2);
    gl::CSum<R> s0, s1, s2;
    for (int j = lane; j < n_int; j += 32) {
      R sn, cs;
      gl::sincospi_<R>(R(2) * (R)j / (R)n_int, &sn, &cs);
      R ff, fl, fq;
      gl::snapped_integrands<R>(rx, ry, dx, dy1, dy2, cs, sn, &ff, &fl, &fq);
      const R w = (j & 1) ? R(4) : R(2);
      s0.add(w * ff);
      s1.add(w * fl);
      s2.add(w * fq);
    }
    double I[3] = {(double)s0.value(), (double)s1.value(), (double)s2.value()};
    for (int o = 16; o > 0; o >>= 1)
      for (int m = 0; m < 3; ++m) I[m] += __shfl_xor_sync(0xffffffffu, I[m], o);
    const double h3 = 2.0 * gl::kPi / n_int / 3.0;
    if (lane == 0)
      out[i] = 1.0 - (c.c0 * I[0] + c.c1 * I[1] + c.c2 * I[2]) * h3 * c.invF0;
  }
}


// ------------------------------------------------------------------ host helpers
// Gauss-Legendre nodes on [-1, 1] by Newton's method on the Legendre recurrence,
// mapped through theta = m + h sin(pi s / 2).
template <typename R>
NodeRule<R> build_rule(int n) {
  NodeRule<R> r;
  memset(&r, 0, sizeof r);
  r.n = n;
  for (int i = 0; i < n; ++i) {
    double z = cos(gl::kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double w = 2.0 / ((1.0 - z * z) * dp * dp);
    double sg = sin(0.5 * gl::kPi * z);
    r.sig[i] = (R)sg;
    r.wt[i] = (R)(w * 0.5 * gl::kPi * cos(0.5 * gl::kPi * z));
    r.cph[i] = (R)cos(gl::kPi * sg);
    r.sph[i] = (R)sin(gl::kPi * sg);
  }
  return r;
}

std::mutex g_dev_mutex;
std::vector<int> g_dev_ready;   // per device: node tables uploaded

cudaError_t ensure_device_tables(int device) {
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  if ((int)g_dev_ready.size() <= device) g_dev_ready.resize(device + 1, 0);
  if (g_dev_ready[device]) return cudaSuccess;
  NodeRule<double> r64 = build_rule<double>(kNodes64);
  NodeRule<double> r64w = build_rule<double>(kNodes64Wide);
  NodeRule<float> r32 = build_rule<float>(kNodes32);
  NodeRule<float> rt[4];
  for (int i = 0; i < 4; ++i) rt[i] = build_rule<float>(kTuneNodes[i]);
  cudaError_t e = cudaMemcpyToSymbol(c_rule64, &r64, sizeof r64);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rule64_wide, &r64w, sizeof r64w);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rule32, &r32, sizeof r32);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rule32_tuned, rt, sizeof rt);
  if (e == cudaSuccess) {
    double inv[65];
    inv[0] = 0.0;
    for (int n = 1; n <= 64; ++n) inv[n] = 1.0 / (double)n;
    e = cudaMemcpyToSymbol(c_inv_n, inv, sizeof inv);
  }
  if (e == cudaSuccess) g_dev_ready[device] = 1;
  return e;
}

}  // namespace

// ------------------------------------------------------------------ context
struct gl_context {
  int device = 0;
  char err[512] = {0};
  SetConst* d_sets = nullptr;
  size_t sets_cap = 0;
  char* d_stage = nullptr;     // staging of host inputs
  size_t stage_cap = 0;
  char* h_stage = nullptr;     // pinned host mirror: host inputs are packed here, one copy
  size_t h_stage_cap = 0;
  cudaEvent_t stage_ev = nullptr;   // recorded after the last copy out of h_stage
  double* d_out = nullptr;     // staging of a host output
  size_t out_cap = 0;
  int* d_status = nullptr;
  unsigned int* d_counter = nullptr;   // tile counter of the persistent kernel
  int sms = 0;
  int occ[16] = {0};                   // resident CTAs per SM by (precision, counting, threads)
  struct LcCfg {
    int threads, tile, cap, rule_idx;
    int qvar;   // item pipeline: quadrature kernel variant (0: MINB = 4, 1: MINB = 8)
    int gvar;   // item pipeline: exposure kernel block (0: 256 threads, 1: 64 threads)
  } cfg[2] = {{256, 256, 1024, -1, 0, 0}, {256, 256, 1024, -1, 0, 0}};   // FP64, FP32C
  struct TuneInfo {
    int tuned = 0, candidates = 0, admissible = 0;
    double best_ms = 0, default_ms = 0, max_err = 0;
  } tune[2];
  // surrogate path workspace (grow-only)
  int64_t sur_cap = 0, sur_rec_cap = 0;
  float *sx = nullptr, *sy = nullptr, *so = nullptr, *sfeat = nullptr, *sscale = nullptr;
  float *sdsph = nullptr, *sthat = nullptr, *sdef = nullptr, *stable = nullptr;
  int *sset = nullptr, *scls = nullptr, *sfb = nullptr, *srj = nullptr, *srns = nullptr,
      *srfirst = nullptr;
  unsigned long long* scount = nullptr;   // items, records, fallback
  double* d_ref = nullptr;             // autotuner: FP64 reference output
  size_t ref_cap = 0;
  double* d_err = nullptr;             // autotuner: max |difference| slot
  unsigned long long* d_counts = nullptr;   // GL_COUNT_* slots
  bool counting = false;
  // item pipeline of the light-curve kernel (grow-only workspace, sized for FP64 items)
  bool item_pipeline = true;
  int64_t item_max = kItemMaxDefault;   // most items one call may queue
  void* d_items = nullptr;
  size_t items_bytes = 0;
  unsigned long long* d_ictr = nullptr;    // kIcWords counter words, zeroed by every step
  // ensemble workspace: parameter sets (12 x n), log prior, log likelihood, light
  // curves (n x n_times), proposals (n/2 x GL_FIT_DIM), z, proposal log posterior,
  // exposure times
  double* d_ens = nullptr;
  size_t ens_cap = 0;
  int qocc[2][2] = {{0, 0}, {0, 0}};       // resident quadrature CTAs per SM (FP64, FP32C) x variant
  int eocc[2][2] = {{0, 0}, {0, 0}};       // resident exposure-kernel CTAs per SM x variant
  int wocc = 0;                            // resident window-kernel CTAs per SM
  // graph cache: one captured step per distinct argument set
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  struct GraphEntry {
    unsigned char key[256];
    size_t key_len;
    cudaGraphExec_t exec;
    cudaGraph_t graph;                 // kept only for profiled steps (their mark nodes)
    cudaGraphNode_t marks[kMarks];     // event-record nodes at the kernel boundaries
    uint64_t last_use;
    int64_t kernels;   // kernel launches in the captured step
  };
  std::vector<GraphEntry> graph_cache;
  uint64_t graph_clock = 0;
  int64_t graph_launches = 0;
  int64_t launches = 0;
  size_t alloc_limit = 0;       // gl_debug_alloc_limit (0: none)
  // per-kernel event timing (gl_profile_enable)
  bool profiling = false;      // mode 1: eager launches bracketed by events
  bool gprof = false;          // mode 2: event-record nodes inside the step graph
  bool capturing = false;      // a step is being captured
  std::vector<cudaEvent_t> ev[GL_KERNEL_KINDS];   // pairs: start, stop
  size_t ev_used[GL_KERNEL_KINDS] = {0};
  cudaEvent_t gmark_cap[kMarks] = {};              // recorded at capture (names the nodes)
  std::vector<std::array<cudaEvent_t, kMarks>> gpool;   // one set per profiled replay
  size_t gpool_used = 0;
};

namespace {

int fail(gl_context* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

#define GL_CUDA(ctx, call)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      return fail((ctx), GL_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    }                                                                                  \
  } while (0)

// true if p is device (or managed) memory usable on `device`
bool is_device_ptr(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == device;
  if (a.type == cudaMemoryTypeManaged) return true;
  return false;
}

void drop_graph(gl_context::GraphEntry& g) {
  cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
}

void drop_graphs(gl_context* ctx) {
  for (auto& g : ctx->graph_cache) drop_graph(g);
  ctx->graph_cache.clear();
}

int grow(gl_context* ctx, void** buf, size_t* cap, size_t need) {
  if (need <= *cap) return GL_OK;
  drop_graphs(ctx);   // captured steps hold the old addresses
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  size_t sz = need + need / 4 + 4096;
  if (ctx->alloc_limit && sz > ctx->alloc_limit)
    return fail(ctx, GL_ENOMEM, "allocation of %zu bytes refused (test limit %zu bytes)", sz,
                ctx->alloc_limit);
  if (cudaMalloc(buf, sz) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, GL_ENOMEM, "cudaMalloc of %zu bytes failed", sz);
  }
  *cap = sz;
  return GL_OK;
}

// Stage a list of input arrays: device arrays pass through, host arrays are
// packed into the pinned mirror ctx->h_stage and sent to ctx->d_stage with one
// copy (one transfer instead of one per array).  `any_host` reports whether a
// copy was made.  The mirror is rewritten only after the previous copy out of it
// has completed.
struct StageItem {
  const void** ptr;
  size_t bytes;
};

int stage_inputs(gl_context* ctx, StageItem* items, int n, cudaStream_t st, bool* any_host) {
  size_t need = 0;
  bool host[64];
  for (int i = 0; i < n; ++i) {
    host[i] = (*items[i].ptr != nullptr) && !is_device_ptr(*items[i].ptr, ctx->device);
    if (host[i]) need += (items[i].bytes + 255) & ~(size_t)255;
  }
  *any_host = false;
  if (need == 0) return GL_OK;
  int rc = grow(ctx, (void**)&ctx->d_stage, &ctx->stage_cap, need);
  if (rc) return rc;
  if (!ctx->stage_ev) GL_CUDA(ctx, cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming));
  GL_CUDA(ctx, cudaEventSynchronize(ctx->stage_ev));   // the mirror is free again
  if (need > ctx->h_stage_cap) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_cap = 0;
    const size_t sz = need + need / 4 + 4096;
    if (cudaMallocHost((void**)&ctx->h_stage, sz) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, GL_ENOMEM, "cudaMallocHost of %zu bytes failed", sz);
    }
    ctx->h_stage_cap = sz;
  }
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    if (!host[i]) continue;
    if (items[i].bytes) memcpy(ctx->h_stage + off, *items[i].ptr, items[i].bytes);
    *items[i].ptr = ctx->d_stage + off;
    off += (items[i].bytes + 255) & ~(size_t)255;
    *any_host = true;
  }
  GL_CUDA(ctx, cudaMemcpyAsync(ctx->d_stage, ctx->h_stage, off, cudaMemcpyHostToDevice, st));
  GL_CUDA(ctx, cudaEventRecord(ctx->stage_ev, st));
  return GL_OK;
}

constexpr size_t kMaxTimed = 65536;

// Record the start event of a launch of `kind` (returns the pair index or -1).
long prof_begin(gl_context* ctx, int kind, cudaStream_t st) {
  if (!ctx->profiling) return -1;
  size_t i = ctx->ev_used[kind];
  if (i >= kMaxTimed) return -1;
  auto& v = ctx->ev[kind];
  if (v.size() < 2 * (i + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    v.push_back(a);
    v.push_back(b);
  }
  cudaEventRecord(v[2 * i], st);
  ctx->ev_used[kind] = i + 1;
  return (long)i;
}

void prof_end(gl_context* ctx, int kind, long i, cudaStream_t st) {
  if (i >= 0) cudaEventRecord(ctx->ev[kind][2 * i + 1], st);
}

// Mode 2: while a step is captured for profiling, record boundary mark k as an
// event-record node of the graph (each replay then points it at its own event).
void gmark(gl_context* ctx, int k, cudaStream_t st) {
  if (ctx->gprof && ctx->capturing && ctx->gmark_cap[k])
    cudaEventRecordWithFlags(ctx->gmark_cap[k], st, cudaEventRecordExternal);
}

int launch_grid(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 148LL * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Carve the item workspace (kItemBytes per item) into the kernels' arrays.
void item_arrays(void* base, int64_t cap, int64_t n_total, size_t rsize, LcArgs* a) {
  char* p = (char*)base;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 255) & ~(size_t)255;
    return q;
  };
  a->ipos = take(3 * rsize * (size_t)cap);
  a->idef = take(rsize * (size_t)cap);
  a->iset = (int*)take(sizeof(int) * (size_t)cap);
  a->iq = (int*)take(sizeof(int) * (size_t)cap);
  a->ihq = (int*)take(sizeof(int) * (size_t)cap);
  a->rj = (int*)take(sizeof(int) * (size_t)cap);
  a->rfirst = (int*)take(sizeof(int) * (size_t)cap);
  a->rns = (int*)take(sizeof(int) * (size_t)cap);
  a->item_cap = cap;
  a->klist = (int*)take(sizeof(int) * (size_t)n_total);
  a->kset = (int*)take(sizeof(int) * (size_t)n_total);
  a->ovlist = (int*)take(sizeof(int) * (size_t)n_total);
}

size_t item_workspace_bytes(int64_t cap, int64_t n_total) {
  return (size_t)cap * kItemBytes + (size_t)n_total * 3 * sizeof(int) + 20 * 256;
}

// Launch of an item-pipeline kernel that depends on the kernel before it in the
// stream: with programmatic stream serialisation (its CTAs are dispatched as that
// kernel's CTAs exit, and wait in pdl_wait), unless profiling puts event records
// between the kernels.
void launch_dependent(gl_context* ctx, void (*k)(LcArgs), int grid, int block, cudaStream_t st,
                      const LcArgs& args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  if (!ctx->profiling && !ctx->gprof) {
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, k, args);
}

// The item pipeline: window tests, kept exposures, quadrature, exposure sums.
template <typename R>
int launch_items(gl_context* ctx, const LcArgs& args, cudaStream_t st) {
  const int qvar = ctx->cfg[sizeof(R) == 4 ? 1 : 0].qvar;
  int& qocc = ctx->qocc[sizeof(R) == 4 ? 1 : 0][qvar];
  const int gvar = ctx->cfg[sizeof(R) == 4 ? 1 : 0].gvar;
  int& eocc = ctx->eocc[sizeof(R) == 4 ? 1 : 0][gvar];
  if (qocc == 0 || eocc == 0 || ctx->wocc == 0) {
    GL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &qocc, qvar ? gl_items_quad_kernel<R, 128, 8> : gl_items_quad_kernel<R, 128, 4>,
                     128, 0));
    GL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &eocc, gvar ? gl_expgeo_kernel<R, 64> : gl_expgeo_kernel<R, 256>,
                     gvar ? 64 : 256, 0));
    GL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->wocc, gl_win_kernel<kWinU>,
                                                               256, 0));
    if (qocc < 1 || eocc < 1 || ctx->wocc < 1)
      return fail(ctx, GL_ECUDA, "item kernels do not fit on an SM");
  }
  // (the counters were zeroed by the setup kernel of this step)
  // window kernel: one pass of 256 x kWinU exposures per block, one wave at most
  // (two exposures per thread and pass measured fastest: a pass that spans a set
  // boundary takes the slower path, and wider passes span more of them)
  int64_t wb = (args.n_total + 256 * kWinU - 1) / (256 * kWinU);
  if (wb > (int64_t)ctx->sms * ctx->wocc) wb = (int64_t)ctx->sms * ctx->wocc;
  if (wb < 1) wb = 1;
  long pe = prof_begin(ctx, GL_KERNEL_WINDOW, st);
  launch_dependent(ctx, gl_win_kernel<kWinU>, (int)wb, 256, st, args);
  prof_end(ctx, GL_KERNEL_WINDOW, pe, st);
  gmark(ctx, kMarkWindow, st);
  pe = prof_begin(ctx, GL_KERNEL_CURVE, st);
  if (gvar)
    launch_dependent(ctx, gl_expgeo_kernel<R, 64>, ctx->sms * eocc, 64, st, args);
  else
    launch_dependent(ctx, gl_expgeo_kernel<R, 256>, ctx->sms * eocc, 256, st, args);
  prof_end(ctx, GL_KERNEL_CURVE, pe, st);
  gmark(ctx, kMarkExposures, st);
  ctx->launches += 2;
  GL_CUDA(ctx, cudaGetLastError());
  pe = prof_begin(ctx, GL_KERNEL_QUAD, st);
  long pq = prof_begin(ctx, GL_KERNEL_ITEMS, st);
  launch_dependent(ctx, qvar ? gl_items_quad_kernel<R, 128, 8> : gl_items_quad_kernel<R, 128, 4>,
                   ctx->sms * qocc, 128, st, args);
  prof_end(ctx, GL_KERNEL_ITEMS, pq, st);
  gmark(ctx, kMarkItems, st);
  // (the 8-CTA quadrature variant marks a large batch: then a full SM of sum
  // threads, whose dependent loads per record need all the parallelism there is)
  launch_dependent(ctx, gl_items_sum_kernel<R>, ctx->sms * (qvar ? 8 : 2), 256, st, args);
  prof_end(ctx, GL_KERNEL_QUAD, pe, st);
  gmark(ctx, kMarkSums, st);
  ctx->launches += 2;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

template <typename R, int NT, bool COUNT>
int launch_lc_nt(gl_context* ctx, LcArgs args, int occ_slot, cudaStream_t st) {
  size_t smem = LcSmem<R>::total(args.tile, args.cap);
  int& occ = ctx->occ[occ_slot];
  if (occ == 0) {
    GL_CUDA(ctx, cudaFuncSetAttribute(gl_lc_kernel<R, NT, COUNT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GL_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gl_lc_kernel<R, NT, COUNT>,
                                                               NT, smem));
    if (occ < 1) return fail(ctx, GL_ECUDA, "light-curve kernel does not fit on an SM");
  }
  int grid = ctx->sms * occ;
  if (grid > args.n_tiles) grid = args.n_tiles;
  if (grid < 1) grid = 1;
  GL_CUDA(ctx, cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), st));
  long pe = prof_begin(ctx, GL_KERNEL_CURVE, st);
  gl_lc_kernel<R, NT, COUNT><<<grid, NT, smem, st>>>(args);
  prof_end(ctx, GL_KERNEL_CURVE, pe, st);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

// occupancy is cached per (precision, counting, threads) instance
bool lc_ready(const gl_context* ctx, int prec, bool items) {
  if (items) {
    const int pi = prec == GL_FP64 ? 0 : 1;
    return ctx->qocc[pi][ctx->cfg[pi].qvar] != 0 && ctx->eocc[pi][ctx->cfg[pi].gvar] != 0 &&
           ctx->wocc != 0;
  }
  const gl_context::LcCfg& cf = ctx->cfg[prec == GL_FP64 ? 0 : 1];
  int slot = (prec == GL_FP64 ? 0 : 1) + (ctx->counting ? 2 : 0) + (cf.threads == 128 ? 4 : 0);
  return ctx->occ[slot] != 0;
}

template <typename R, bool COUNT>
int launch_lc(gl_context* ctx, const LcArgs& args0, cudaStream_t st) {
  const gl_context::LcCfg& cf = ctx->cfg[sizeof(R) == 4 ? 1 : 0];
  LcArgs args = args0;
  args.tile = cf.tile;
  args.cap = cf.cap;
  args.rule_idx = cf.rule_idx;
  args.n_tiles = (int)((args.n_total + cf.tile - 1) / cf.tile);
  args.tile_counter = ctx->d_counter;
  args.counts = ctx->d_counts;
  if (args.ipos && !COUNT) return launch_items<R>(ctx, args, st);
  int slot = (sizeof(R) == 4 ? 1 : 0) + (COUNT ? 2 : 0) + (cf.threads == 128 ? 4 : 0);
  if (cf.threads == 128) return launch_lc_nt<R, 128, COUNT>(ctx, args, slot, st);
  return launch_lc_nt<R, 256, COUNT>(ctx, args, slot, st);
}

// One light-curve step: per-set constants, then the fused kernel (and, with the
// item pipeline, its quadrature and exposure-sum stages).
struct StepArgs {
  ParamPtrs pp;
  int64_t n_sets;
  const int64_t* offsets;
  const double* t;
  int64_t n_times, n_total;
  double* out;
  int prec;
  SetConst* sets;
  void* items;        // item workspace, or null: every tile integrates locally
  int64_t item_cap;
  int locked;         // tidally locked bodies: gl_locked_kernel
  int gprof;          // captured with boundary marks (profiling mode 2)
};

int enqueue_step(gl_context* ctx, const StepArgs& sa, cudaStream_t st) {
  NvtxRange nv("light-curve step: enqueue kernels");
  gmark(ctx, kMarkStart, st);
  long pe = prof_begin(ctx, GL_KERNEL_SETUP, st);
  // the item pipeline's counters are zeroed here (one graph node less than a
  // separate memset)
  const bool pipeline = sa.items && !sa.locked && !ctx->counting;
  gl_setup_kernel<<<(int)((sa.n_sets + 31) / 32), 128, 0, st>>>(
      sa.pp, sa.n_sets, sa.offsets, sa.n_total, sa.sets, ctx->d_status,
      pipeline ? ctx->d_ictr : nullptr, pipeline ? (int)kIcWords : 0);
  prof_end(ctx, GL_KERNEL_SETUP, pe, st);
  gmark(ctx, kMarkSetup, st);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  LcArgs la;
  memset(&la, 0, sizeof la);
  la.sets = sa.sets;
  la.t = sa.t;
  la.offsets = sa.offsets;
  la.n_times = sa.n_times;
  la.n_sets = sa.n_sets;
  la.n_total = sa.n_total;
  la.out = sa.out;
  if (sa.locked) {
    const int rule_idx = ctx->cfg[sa.prec == GL_FP64 ? 0 : 1].rule_idx;
    pe = prof_begin(ctx, GL_KERNEL_CURVE, st);
    const int grid = launch_grid(sa.n_total, 128);
    if (sa.prec == GL_FP64)
      gl_locked_kernel<double><<<grid, 128, 0, st>>>(sa.sets, sa.t, sa.offsets, sa.n_times,
                                                     sa.n_sets, sa.n_total, rule_idx, sa.out);
    else
      gl_locked_kernel<float><<<grid, 128, 0, st>>>(sa.sets, sa.t, sa.offsets, sa.n_times,
                                                    sa.n_sets, sa.n_total, rule_idx, sa.out);
    prof_end(ctx, GL_KERNEL_CURVE, pe, st);
    ctx->launches++;
    GL_CUDA(ctx, cudaGetLastError());
    return GL_OK;
  }
  if (sa.items) {
    item_arrays(sa.items, sa.item_cap, sa.n_total, sa.prec == GL_FP64 ? sizeof(double) : sizeof(float),
                &la);
    la.ictr = ctx->d_ictr;
    la.n_smsp = 4 * ctx->sms;
  }
  if (sa.prec == GL_FP64)
    return ctx->counting ? launch_lc<double, true>(ctx, la, st) : launch_lc<double, false>(ctx, la, st);
  return ctx->counting ? launch_lc<float, true>(ctx, la, st) : launch_lc<float, false>(ctx, la, st);
}

// Replay a captured step for these exact arguments, capturing it on first use.
// Capture happens on the context's private stream; the graph is launched on `st`.
int launch_step_graph(gl_context* ctx, const StepArgs& sa, cudaStream_t st) {
  NvtxRange nv("light-curve step: graph");
  unsigned char key[sizeof(StepArgs)];
  memcpy(key, &sa, sizeof sa);
  gl_context::GraphEntry* hit = nullptr;
  for (auto& g : ctx->graph_cache)
    if (g.key_len == sizeof key && memcmp(g.key, key, sizeof key) == 0) hit = &g;
  if (!hit) {
    // the occupancy query and attribute setting must not happen inside a capture
    if (!sa.locked && !lc_ready(ctx, sa.prec, sa.items != nullptr))
      return enqueue_step(ctx, sa, st);   // first call: eager
    if (sa.gprof)
      for (int k = 0; k < kMarks; ++k)
        if (!ctx->gmark_cap[k]) GL_CUDA(ctx, cudaEventCreate(&ctx->gmark_cap[k]));
    GL_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int64_t l0 = ctx->launches;
    ctx->capturing = true;
    int rc = enqueue_step(ctx, sa, ctx->cap_stream);
    ctx->capturing = false;
    const int64_t kernels = ctx->launches - l0;
    ctx->launches = l0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(ctx, GL_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
    gl_context::GraphEntry ge;
    memset(&ge, 0, sizeof ge);
    if (sa.gprof) {
      // find the boundary marks among the graph's nodes by the event each records
      size_t nn = 0;
      cudaGraphGetNodes(graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord)
          continue;
        cudaEvent_t ev = nullptr;
        if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
        for (int k = 0; k < kMarks; ++k)
          if (ev == ctx->gmark_cap[k]) ge.marks[k] = nodes[i];
      }
      cudaGetLastError();
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (sa.gprof) ge.graph = graph;
    else cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      if (ge.graph) cudaGraphDestroy(ge.graph);
      return fail(ctx, GL_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    if (ctx->graph_cache.size() >= 16) {
      size_t lru = 0;
      for (size_t i = 1; i < ctx->graph_cache.size(); ++i)
        if (ctx->graph_cache[i].last_use < ctx->graph_cache[lru].last_use) lru = i;
      drop_graph(ctx->graph_cache[lru]);
      ctx->graph_cache.erase(ctx->graph_cache.begin() + lru);
    }
    memcpy(ge.key, key, sizeof key);
    ge.key_len = sizeof key;
    ge.exec = exec;
    ge.last_use = 0;
    ge.kernels = kernels;
    ctx->graph_cache.push_back(ge);
    hit = &ctx->graph_cache.back();
  }
  hit->last_use = ++ctx->graph_clock;
  if (sa.gprof && ctx->gpool_used < kMaxTimed) {
    // this replay's marks record into a fresh set of events
    if (ctx->gpool.size() <= ctx->gpool_used) {
      std::array<cudaEvent_t, kMarks> evs{};
      for (int k = 0; k < kMarks; ++k) GL_CUDA(ctx, cudaEventCreate(&evs[k]));
      ctx->gpool.push_back(evs);
    }
    const auto& evs = ctx->gpool[ctx->gpool_used];
    for (int k = 0; k < kMarks; ++k)
      if (hit->marks[k])
        GL_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(hit->exec, hit->marks[k], evs[k]));
    ctx->gpool_used++;
  }
  GL_CUDA(ctx, cudaGraphLaunch(hit->exec, st));
  ctx->launches += hit->kernels;
  ctx->graph_launches++;
  return GL_OK;
}

}  // namespace

extern "C" {

int gl_context_create(gl_context** out, int device) {
  if (!out) return GL_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return GL_ECUDA;
  }
  if (device < 0 || device >= ndev) return GL_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return GL_ECUDA;
  if (ensure_device_tables(device) != cudaSuccess) return GL_ECUDA;
  gl_context* ctx = new gl_context();
  ctx->device = device;
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_counter, sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_counts, GL_COUNT_SLOTS * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->d_counts, 0, GL_COUNT_SLOTS * sizeof(unsigned long long)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return GL_ECUDA;
  }
  *out = ctx;
  return GL_OK;
}

int gl_context_destroy(gl_context* ctx) {
  if (!ctx) return GL_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->d_sets) cudaFree(ctx->d_sets);
  if (ctx->d_stage) cudaFree(ctx->d_stage);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
  if (ctx->d_out) cudaFree(ctx->d_out);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_counter) cudaFree(ctx->d_counter);
  if (ctx->d_counts) cudaFree(ctx->d_counts);
  if (ctx->d_ref) cudaFree(ctx->d_ref);
  if (ctx->d_items) cudaFree(ctx->d_items);
  if (ctx->d_ens) cudaFree(ctx->d_ens);
  if (ctx->d_ictr) cudaFree(ctx->d_ictr);
  for (void* q : {(void*)ctx->sx, (void*)ctx->sy, (void*)ctx->so, (void*)ctx->sfeat,
                  (void*)ctx->sscale, (void*)ctx->sdsph, (void*)ctx->sthat, (void*)ctx->sdef,
                  (void*)ctx->stable, (void*)ctx->sset, (void*)ctx->scls, (void*)ctx->sfb,
                  (void*)ctx->srj, (void*)ctx->srns, (void*)ctx->srfirst, (void*)ctx->scount})
    if (q) cudaFree(q);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (auto& g : ctx->graph_cache) cudaGraphExecDestroy(g.exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (int k = 0; k < GL_KERNEL_KINDS; ++k)
    for (cudaEvent_t e : ctx->ev[k]) cudaEventDestroy(e);
  delete ctx;
  return GL_OK;
}

const char* gl_last_error(const gl_context* ctx) { return ctx ? ctx->err : "no context"; }

int64_t gl_launch_count(const gl_context* ctx) { return ctx ? ctx->launches : 0; }

int gl_counts_enable(gl_context* ctx, int on) {
  if (!ctx) return GL_EINVAL;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  GL_CUDA(ctx, cudaMemset(ctx->d_counts, 0, GL_COUNT_SLOTS * sizeof(unsigned long long)));
  ctx->counting = on != 0;
  return GL_OK;
}

int gl_counts_read(gl_context* ctx, int64_t* counts, int n) {
  if (!ctx || !counts || n < 0) return GL_EINVAL;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  GL_CUDA(ctx, cudaDeviceSynchronize());
  unsigned long long h[GL_COUNT_SLOTS];
  GL_CUDA(ctx, cudaMemcpy(h, ctx->d_counts, sizeof h, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n && i < GL_COUNT_SLOTS; ++i) counts[i] = (int64_t)h[i];
  for (int i = GL_COUNT_SLOTS; i < n; ++i) counts[i] = 0;
  return GL_OK;
}

int gl_graphs_enable(gl_context* ctx, int on) {
  if (!ctx) return GL_EINVAL;
  ctx->graphs = on != 0;
  if (!ctx->graphs) drop_graphs(ctx);
  return GL_OK;
}

int64_t gl_graph_launches(const gl_context* ctx) { return ctx ? ctx->graph_launches : 0; }

int gl_item_pipeline(gl_context* ctx, int on, int64_t max_items) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (max_items < 0 || max_items >= (1LL << 31)) return fail(ctx, GL_EINVAL, "max_items out of range");
  ctx->item_pipeline = on != 0;
  ctx->item_max = max_items > 0 ? max_items : kItemMaxDefault;
  drop_graphs(ctx);
  return GL_OK;
}

int gl_configure(gl_context* ctx, gl_precision prec, int threads, int nodes, int quad_ctas,
                 int exposure_block) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision");
  if (threads != 0 && threads != 128 && threads != 256)
    return fail(ctx, GL_EINVAL, "threads must be 0, 128 or 256");
  if (quad_ctas != 0 && quad_ctas != 4 && quad_ctas != 8)
    return fail(ctx, GL_EINVAL, "quad_ctas must be 0, 4 or 8");
  if (exposure_block != 0 && exposure_block != 64 && exposure_block != 256)
    return fail(ctx, GL_EINVAL, "exposure_block must be 0, 64 or 256");
  int ni = -1;
  if (nodes != 0) {
    if (prec == GL_FP64) return fail(ctx, GL_EINVAL, "the FP64 path has a fixed order");
    for (int i = 0; i < 4; ++i)
      if (kTuneNodes[i] == nodes) ni = i;
    if (ni < 0) return fail(ctx, GL_EINVAL, "nodes must be 0, 16, 20, 24 or 28");
  }
  const int th = threads ? threads : 256;
  ctx->cfg[prec == GL_FP64 ? 0 : 1] = {th, th, 4 * th, ni, quad_ctas == 8 ? 1 : 0,
                                       exposure_block == 64 ? 1 : 0};
  drop_graphs(ctx);
  return GL_OK;
}

int gl_autotune(gl_context* ctx, const gl_params* p, const gl_times* tm, double* out,
                gl_precision prec, void* stream, gl_tune_report* rep) {
  NvtxRange nv("gl_autotune");
  if (!ctx || !p || !tm || !out) return GL_EINVAL;
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision");
  if (!is_device_ptr(out, ctx->device) || !is_device_ptr(tm->t, ctx->device))
    return fail(ctx, GL_EINVAL, "autotuning needs device buffers");
  if (tm->n_total <= 0 || p->n_sets <= 0) return fail(ctx, GL_EINVAL, "empty batch");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  bool was_prof = ctx->profiling, was_count = ctx->counting, was_graph = ctx->graphs;
  ctx->profiling = false;
  ctx->counting = false;
  // candidates are timed the way later calls run: as CUDA-graph replays when
  // graphs are on (each candidate captures its own graph)
  ctx->graphs = false;
  drop_graphs(ctx);
  int rc = grow(ctx, (void**)&ctx->d_ref, &ctx->ref_cap, (size_t)tm->n_total * sizeof(double));
  if (rc) return rc;
  if (!ctx->d_err) GL_CUDA(ctx, cudaMalloc(&ctx->d_err, sizeof(unsigned long long)));
  // reference: the FP64 path with its default configuration
  gl_context::LcCfg saved[2] = {ctx->cfg[0], ctx->cfg[1]};
  ctx->cfg[0] = {256, 256, 1024, -1, 0, 0};
  rc = gl_lightcurve_batch(ctx, p, tm, ctx->d_ref, GL_FP64, stream);
  if (rc) return rc;
  const int pi = prec == GL_FP64 ? 0 : 1;
  const double tol = prec == GL_FP64 ? 1e-10 : 1e-7;
  // The second axis is the tile kernel's CTA size, or with the item pipeline
  // (whose launch shapes are fixed) the quadrature kernel's variant.
  struct Cand { int threads, nodes_idx, qvar, gvar; };
  Cand cands[16];
  int nc = 0;
  for (int gv = 0; gv < (ctx->item_pipeline ? 2 : 1); ++gv) {
    for (int ax = 0; ax < 2; ++ax) {
      const int th = ctx->item_pipeline ? 256 : (ax ? 256 : 128);
      const int qv = ctx->item_pipeline ? ax : 0;
      if (prec == GL_FP64) {
        cands[nc++] = {th, -1, qv, gv};
      } else {
        for (int ni = 0; ni < 4; ++ni) cands[nc++] = {th, ni, qv, gv};
      }
    }
  }
  cudaEvent_t e0, e1;
  GL_CUDA(ctx, cudaEventCreate(&e0));
  GL_CUDA(ctx, cudaEventCreate(&e1));
  // Each timed run starts from a cold L2 (a buffer twice its size is written
  // first, outside the events): the conservative case, and the way benchmarks
  // time a step.  Without room for the buffer the runs are timed warm.
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
  const size_t flush_bytes = 2 * (size_t)(l2 > 0 ? l2 : 0);
  void* flush = nullptr;
  if (flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  double best_ms = 1e30, default_ms = 0.0, best_err = 0.0;
  int best = -1, admissible = 0;
  for (int ci = 0; ci < nc && rc == GL_OK; ++ci) {
    ctx->cfg[pi] = {cands[ci].threads, cands[ci].threads, 4 * cands[ci].threads,
                    cands[ci].nodes_idx, cands[ci].qvar, cands[ci].gvar};
    drop_graphs(ctx);
    ctx->graphs = was_graph;
    rc = gl_lightcurve_batch(ctx, p, tm, out, prec, stream);
    if (rc) break;
    cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned long long), st);
    gl_maxdiff_kernel<<<ctx->sms * 4, 256, 0, st>>>(out, ctx->d_ref, tm->n_total,
                                                     (unsigned long long*)ctx->d_err);
    unsigned long long eb = 0;
    cudaMemcpyAsync(&eb, ctx->d_err, sizeof eb, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(ctx, GL_ECUDA, "autotune synchronisation failed");
      break;
    }
    double err;
    memcpy(&err, &eb, sizeof err);
    bool ok = err <= 0.9 * tol;
    float ms = 1e30f;
    if (ok) {
      ++admissible;
      for (int rep_i = 0; rep_i < 5; ++rep_i) {
        if (flush) cudaMemsetAsync(flush, rep_i & 0xff, flush_bytes, st);
        cudaEventRecord(e0, st);
        rc = gl_lightcurve_batch(ctx, p, tm, out, prec, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float m = 0.f;
        cudaEventElapsedTime(&m, e0, e1);
        if (m < ms) ms = m;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = ci;
        best_err = err;
      }
    }
    if (cands[ci].threads == 256 && cands[ci].qvar == 0 && cands[ci].gvar == 0 &&
        (cands[ci].nodes_idx == 1 || cands[ci].nodes_idx == -1))
      default_ms = ok ? ms : 0.0;
    ctx->graphs = false;
    drop_graphs(ctx);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) {
    cudaStreamSynchronize(st);
    cudaFree(flush);
  }
  ctx->cfg[0] = saved[0];
  ctx->cfg[1] = saved[1];
  if (best >= 0)
    ctx->cfg[pi] = {cands[best].threads, cands[best].threads, 4 * cands[best].threads,
                    cands[best].nodes_idx, cands[best].qvar, cands[best].gvar};
  ctx->profiling = was_prof;
  ctx->counting = was_count;
  ctx->graphs = was_graph;
  drop_graphs(ctx);
  if (rc) return rc;
  if (best < 0) return fail(ctx, GL_ENUMERIC, "no candidate met the tolerance");
  gl_context::TuneInfo& ti = ctx->tune[pi];
  ti.tuned = 1;
  ti.candidates = nc;
  ti.admissible = admissible;
  ti.best_ms = best_ms;
  ti.default_ms = default_ms;
  ti.max_err = best_err;
  if (rep) {
    rep->threads = cands[best].threads;
    rep->tile = cands[best].threads;
    rep->nodes = prec == GL_FP64 ? kNodes64 : kTuneNodes[cands[best].nodes_idx];
    rep->ms = best_ms;
    rep->default_ms = default_ms;
    rep->max_abs_err = best_err;
    rep->candidates = nc;
    rep->admissible = admissible;
    rep->quad_ctas_per_sm =
        ctx->item_pipeline ? ctx->qocc[pi][cands[best].qvar] : 0;
    rep->exposure_block = ctx->item_pipeline ? (cands[best].gvar ? 64 : 256) : 0;
  }
  return GL_OK;
}

int gl_debug_alloc_limit(gl_context* ctx, int64_t bytes) {
  if (!ctx || bytes < 0) return GL_EINVAL;
  ctx->alloc_limit = (size_t)bytes;
  return GL_OK;
}

int gl_profile_enable(gl_context* ctx, int on) {
  if (!ctx || on < 0 || on > 2) return GL_EINVAL;
  ctx->profiling = on == 1;
  ctx->gprof = on == 2;
  for (int k = 0; k < GL_KERNEL_KINDS; ++k) ctx->ev_used[k] = 0;
  ctx->gpool_used = 0;
  return GL_OK;
}

int gl_profile_read(gl_context* ctx, int kind, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches || kind < 0 || kind >= GL_KERNEL_KINDS) return GL_EINVAL;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  double tot = 0.0;
  if (ctx->gprof) {
    // graph replays: the span between the kind's two boundary marks
    int a = -1, b = -1;
    switch (kind) {
      case GL_KERNEL_SETUP: a = kMarkStart; b = kMarkSetup; break;
      case GL_KERNEL_WINDOW: a = kMarkSetup; b = kMarkWindow; break;
      case GL_KERNEL_CURVE: a = kMarkWindow; b = kMarkExposures; break;
      case GL_KERNEL_QUAD: a = kMarkExposures; b = kMarkSums; break;
      case GL_KERNEL_ITEMS: a = kMarkExposures; b = kMarkItems; break;
      case GL_KERNEL_STEP: a = kMarkStart; b = kMarkSums; break;
      default: break;
    }
    int64_t n = 0;
    if (a >= 0)
      for (size_t i = 0; i < ctx->gpool_used; ++i) {
        GL_CUDA(ctx, cudaEventSynchronize(ctx->gpool[i][b]));
        float m = 0.f;
        GL_CUDA(ctx, cudaEventElapsedTime(&m, ctx->gpool[i][a], ctx->gpool[i][b]));
        tot += m;
        ++n;
      }
    *ms = tot;
    *launches = n;
    return GL_OK;
  }
  for (size_t i = 0; i < ctx->ev_used[kind]; ++i) {
    GL_CUDA(ctx, cudaEventSynchronize(ctx->ev[kind][2 * i + 1]));
    float m = 0.f;
    GL_CUDA(ctx, cudaEventElapsedTime(&m, ctx->ev[kind][2 * i], ctx->ev[kind][2 * i + 1]));
    tot += m;
  }
  *ms = tot;
  *launches = (int64_t)ctx->ev_used[kind];
  return GL_OK;
}

int gl_q_to_u(int64_t n, const double* q1, const double* q2, double* u1, double* u2) {
  if (n < 0 || (n > 0 && (!q1 || !q2 || !u1 || !u2))) return GL_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    double s = sqrt(q1[i]);
    u1[i] = 2.0 * s * q2[i];
    u2[i] = s * (1.0 - 2.0 * q2[i]);
  }
  return GL_OK;
}

int gl_sync(gl_context* ctx, void* stream) {
  if (!ctx) return GL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  GL_CUDA(ctx, cudaStreamSynchronize(st));
  int h = 0;
  GL_CUDA(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  GL_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  if (h & kStatusTimeout) return fail(ctx, GL_ETIMEOUT, "a bounded device wait gave up");
  if (h & kStatusBadOffsets) return fail(ctx, GL_EINVAL, "offsets are not a valid CSR index");
  if (h & kStatusInvalidSet) return fail(ctx, GL_ENUMERIC, "a parameter set is physically invalid");
  return GL_OK;
}

}  // extern "C"

namespace {

int lightcurve_impl(gl_context* ctx, const gl_params* p, const gl_times* tm, double* out,
                    gl_precision prec, void* stream, bool locked) {
  NvtxRange nv(locked ? "gl_lightcurve_locked" : "gl_lightcurve_batch");
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (!p || !tm) return fail(ctx, GL_EINVAL, "NULL params or times");
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision %d", (int)prec);
  int64_t n_sets = p->n_sets;
  if (n_sets < 0) return fail(ctx, GL_EINVAL, "n_sets < 0");
  if (tm->n_total < 0 || tm->n_total >= (1LL << 31)) return fail(ctx, GL_EINVAL, "n_total out of range");
  if (!tm->offsets) {
    if (tm->n_times < 0) return fail(ctx, GL_EINVAL, "n_times < 0");
    if (tm->n_total != n_sets * tm->n_times)
      return fail(ctx, GL_EINVAL, "n_total != n_sets * n_times for a shared grid");
  }
  if (!tm->nsuper && tm->nsuper_all < 1) return fail(ctx, GL_EINVAL, "nsuper_all < 1");
  if (n_sets == 0 || tm->n_total == 0) return GL_OK;
  const double* arr[12] = {p->t0, p->period, p->a_rs, p->b, p->ecc, p->omega,
                           p->k, p->f, p->eta, p->xi, p->u1, p->u2};
  for (int i = 0; i < 12; ++i)
    if (!arr[i]) return fail(ctx, GL_EINVAL, "NULL parameter array %d", i);
  if (!tm->t || !tm->exptime || !out) return fail(ctx, GL_EINVAL, "NULL times, exptime or out");
  if (tm->offsets && !is_device_ptr(tm->offsets, ctx->device) &&
      (tm->offsets[0] != 0 || tm->offsets[n_sets] != tm->n_total))
    return fail(ctx, GL_EINVAL, "offsets[0] != 0 or offsets[n_sets] != n_total");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;

  ParamPtrs pp;
  memset(&pp, 0, sizeof pp);   // the struct's bytes key the graph cache
  pp.t0 = p->t0;
  pp.period = p->period;
  pp.a_rs = p->a_rs;
  pp.b = p->b;
  pp.ecc = p->ecc;
  pp.omega = p->omega;
  pp.k = p->k;
  pp.f = p->f;
  pp.eta = p->eta;
  pp.xi = p->xi;
  pp.u1 = p->u1;
  pp.u2 = p->u2;
  pp.g = p->g;
  pp.zeta = p->zeta;
  pp.exptime = tm->exptime;
  pp.nsuper = tm->nsuper;
  pp.nsuper_all = tm->nsuper_all;
  const double* t = tm->t;
  const int64_t* offsets = tm->offsets;
  int64_t n_t = offsets ? tm->n_total : tm->n_times;
  size_t sb = (size_t)n_sets * sizeof(double);
  StageItem items[] = {
      {(const void**)&pp.t0, sb}, {(const void**)&pp.period, sb}, {(const void**)&pp.a_rs, sb},
      {(const void**)&pp.b, sb}, {(const void**)&pp.ecc, sb}, {(const void**)&pp.omega, sb},
      {(const void**)&pp.k, sb}, {(const void**)&pp.f, sb}, {(const void**)&pp.eta, sb},
      {(const void**)&pp.xi, sb}, {(const void**)&pp.u1, sb}, {(const void**)&pp.u2, sb},
      {(const void**)&pp.exptime, sb},
      {(const void**)&pp.nsuper, (size_t)n_sets * sizeof(int32_t)},
      {(const void**)&t, (size_t)n_t * sizeof(double)},
      {(const void**)&offsets, (size_t)(n_sets + 1) * sizeof(int64_t)},
      {(const void**)&pp.g, sb}, {(const void**)&pp.zeta, sb},
  };
  bool any_host = false;
  int rc = stage_inputs(ctx, items, (int)(sizeof items / sizeof items[0]), st, &any_host);
  if (rc) return rc;
  rc = grow(ctx, (void**)&ctx->d_sets, &ctx->sets_cap, (size_t)n_sets * sizeof(SetConst));
  if (rc) return rc;
  bool out_host = !is_device_ptr(out, ctx->device);
  double* d_out = out;
  if (out_host) {
    rc = grow(ctx, (void**)&ctx->d_out, &ctx->out_cap, (size_t)tm->n_total * sizeof(double));
    if (rc) return rc;
    d_out = ctx->d_out;
  }
  void* iws = nullptr;
  int64_t item_cap = 0;
  if (ctx->item_pipeline && !locked) {
    // sized for every sub-exposure of the batch (per-set nsuper: 16 per exposure),
    // capped at item_max; tiles whose items do not fit integrate locally
    int64_t per = tm->nsuper ? 16 : tm->nsuper_all;
    item_cap = tm->n_total > ctx->item_max / per ? ctx->item_max : tm->n_total * per;
    rc = grow(ctx, &ctx->d_items, &ctx->items_bytes, item_workspace_bytes(item_cap, tm->n_total));
    if (rc) return rc;
    if (!ctx->d_ictr)
      GL_CUDA(ctx, cudaMalloc(&ctx->d_ictr, kIcWords * sizeof(unsigned long long)));
    iws = ctx->d_items;
  }
  StepArgs sa;
  memset(&sa, 0, sizeof sa);
  sa.locked = locked ? 1 : 0;
  if (locked) {
    iws = nullptr;
    item_cap = 0;
  }
  sa.items = iws;
  sa.item_cap = item_cap;
  sa.pp = pp;
  sa.n_sets = n_sets;
  sa.offsets = offsets;
  sa.t = t;
  sa.n_times = tm->n_times;
  sa.n_total = tm->n_total;
  sa.out = d_out;
  sa.prec = (int)prec;
  sa.sets = ctx->d_sets;
  // host buffers are staged at fixed device addresses, so their steps replay a
  // graph too (the copies are ordered around it on the stream)
  sa.gprof = ctx->gprof ? 1 : 0;
  bool use_graph = ctx->graphs && !ctx->profiling && !ctx->counting;
  if (use_graph) {
    rc = launch_step_graph(ctx, sa, st);
  } else {
    rc = enqueue_step(ctx, sa, st);
  }
  if (rc) return rc;
  if (out_host) {
    GL_CUDA(ctx, cudaMemcpyAsync(out, d_out, (size_t)tm->n_total * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  }
  if (out_host || any_host) GL_CUDA(ctx, cudaStreamSynchronize(st));
  return GL_OK;
}

}  // namespace

extern "C" {

int gl_lightcurve_batch(gl_context* ctx, const gl_params* p, const gl_times* tm, double* out,
                        gl_precision prec, void* stream) {
  return lightcurve_impl(ctx, p, tm, out, prec, stream, false);
}

int gl_lightcurve_locked(gl_context* ctx, const gl_params* p, const gl_times* tm, double* out,
                         gl_precision prec, void* stream) {
  return lightcurve_impl(ctx, p, tm, out, prec, stream, true);
}

int gl_flux_sphere(gl_context* ctx, int64_t n, const double* x0, const double* y0,
                   const double* z, const double* p, const double* u1, const double* u2,
                   double* out, gl_precision prec, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision %d", (int)prec);
  if (n == 0) return GL_OK;
  if (!x0 || !y0 || !z || !p || !u1 || !u2 || !out) return fail(ctx, GL_EINVAL, "NULL array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  SpherePtrs sp = {x0, y0, z, p, u1, u2};
  size_t b = (size_t)n * sizeof(double);
  StageItem items[] = {{(const void**)&sp.x0, b}, {(const void**)&sp.y0, b},
                       {(const void**)&sp.z, b},  {(const void**)&sp.p, b},
                       {(const void**)&sp.u1, b}, {(const void**)&sp.u2, b}};
  bool any_host = false;
  int rc = stage_inputs(ctx, items, 6, st, &any_host);
  if (rc) return rc;
  bool out_host = !is_device_ptr(out, ctx->device);
  double* d_out = out;
  if (out_host) {
    rc = grow(ctx, (void**)&ctx->d_out, &ctx->out_cap, b);
    if (rc) return rc;
    d_out = ctx->d_out;
  }
  int grid = launch_grid(n, 256);
  long pe = prof_begin(ctx, GL_KERNEL_SPHERE, st);
  if (prec == GL_FP64)
    gl_sphere_kernel<double><<<grid, 256, 0, st>>>(sp, n, d_out, ctx->d_status);
  else
    gl_sphere_kernel<float><<<grid, 256, 0, st>>>(sp, n, d_out, ctx->d_status);
  prof_end(ctx, GL_KERNEL_SPHERE, pe, st);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  if (out_host) GL_CUDA(ctx, cudaMemcpyAsync(out, d_out, b, cudaMemcpyDeviceToHost, st));
  if (out_host || any_host) GL_CUDA(ctx, cudaStreamSynchronize(st));
  return GL_OK;
}

int gl_surrogate_features(gl_context* ctx, int64_t n, const double* x0, const double* y0,
                          const double* k, const double* f, const double* eta, const double* xi,
                          const double* u1, const double* u2, float* feat, float* scale,
                          double* r_area, int32_t* bin, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (n == 0) return GL_OK;
  const void* ptrs[12] = {x0, y0, k, f, eta, xi, u1, u2, feat, scale, r_area, bin};
  for (const void* q : ptrs)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  gl_sur_geom_features_kernel<<<launch_grid(n, 256), 256, 0, (cudaStream_t)stream>>>(
      n, x0, y0, k, f, eta, xi, u1, u2, feat, scale, r_area, bin);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

int gl_surrogate_targets(gl_context* ctx, int64_t n, const double* f_oblate,
                         const double* f_sphere, const float* scale, float* t, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (n == 0) return GL_OK;
  const void* ptrs[4] = {f_oblate, f_sphere, scale, t};
  for (const void* q : ptrs)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  gl_sur_targets_kernel<<<launch_grid(n, 256), 256, 0, (cudaStream_t)stream>>>(n, f_oblate, f_sphere,
                                                                                scale, t);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

int gl_loglike(gl_context* ctx, int64_t n_sets, int64_t n_times, const double* flux,
               const double* data, const double* sigma, double* loglike, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n_sets < 0 || n_times < 0) return fail(ctx, GL_EINVAL, "negative size");
  if (n_sets == 0) return GL_OK;
  const void* ptrs[4] = {flux, data, sigma, loglike};
  for (const void* q : ptrs)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  if (n_sets > 2147483647LL) return fail(ctx, GL_EINVAL, "too many sets");
  gl_loglike_kernel<<<(unsigned)n_sets, 256, 0, (cudaStream_t)stream>>>(n_sets, n_times, flux, data,
                                                                        sigma, loglike);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

static int munu_op(gl_context* ctx, int op, int64_t n, const double* a, const double* b, double* c,
                   double* d, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (n == 0) return GL_OK;
  const void* ptrs[4] = {a, b, c, d};
  for (const void* q : ptrs)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  gl_munu_kernel<<<launch_grid(n, 256), 256, 0, (cudaStream_t)stream>>>(op, n, a, b, c, d);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

int gl_munu_to_feta(gl_context* ctx, int64_t n, const double* mu, const double* nu, double* f,
                    double* eta, void* stream) {
  return munu_op(ctx, kMunuToFeta, n, mu, nu, f, eta, stream);
}

int gl_feta_to_munu(gl_context* ctx, int64_t n, const double* f, const double* eta, double* mu,
                    double* nu, void* stream) {
  return munu_op(ctx, kFetaToMunu, n, f, eta, mu, nu, stream);
}

int gl_munu_prior(gl_context* ctx, int64_t n, const double* u, const double* w, double* mu,
                  double* nu, void* stream) {
  return munu_op(ctx, kMunuPrior, n, u, w, mu, nu, stream);
}

// Log posteriors of m fit vectors into lp (workspace layout of ensure_ensemble).
static int ens_logpost(gl_context* ctx, const gl_ensemble* e, const double* x, int64_t m,
                       double* lp, cudaStream_t st) {
  double* soa = ctx->d_ens;
  double* prior = soa + 12 * e->n_walkers;
  double* ll = prior + e->n_walkers;
  double* flux = ll + e->n_walkers;
  double* exptime = flux + e->n_walkers * e->n_times + (e->n_walkers / 2) * (GL_FIT_DIM + 2);
  const int g = launch_grid(m, 256);
  gl_ens_params_kernel<<<g, 256, 0, st>>>(x, m, e->lo, e->hi, soa, prior);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  gl_params p;
  memset(&p, 0, sizeof p);
  p.n_sets = m;
  const double** f[12] = {&p.t0, &p.period, &p.a_rs, &p.b, &p.ecc, &p.omega,
                          &p.k,  &p.f,      &p.eta,  &p.xi, &p.u1, &p.u2};
  for (int q = 0; q < 12; ++q) *f[q] = soa + q * m;
  gl_times tm;
  memset(&tm, 0, sizeof tm);
  tm.t = e->t;
  tm.n_times = e->n_times;
  tm.n_total = m * e->n_times;
  tm.exptime = exptime;
  tm.nsuper_all = e->nsuper;
  int rc = gl_lightcurve_batch(ctx, &p, &tm, flux, e->prec, st);
  if (rc) return rc;
  gl_loglike_kernel<<<(unsigned)m, 256, 0, st>>>(m, e->n_times, flux, e->data, e->sigma, ll);
  gl_ens_post_kernel<<<g, 256, 0, st>>>(m, prior, ll, lp);
  ctx->launches += 2;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

static int ensure_ensemble(gl_context* ctx, const gl_ensemble* e, cudaStream_t st) {
  if (!e || e->n_walkers < 4 || (e->n_walkers & 1) || e->n_walkers > (1LL << 26))
    return fail(ctx, GL_EINVAL, "n_walkers must be even, in [4, 2^26]");
  if (e->n_times < 1 || e->nsuper < 1 || !(e->exptime >= 0.0) || !(e->a > 1.0))
    return fail(ctx, GL_EINVAL, "bad n_times, nsuper, exptime or stretch scale");
  if (e->prec != GL_FP64 && e->prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision");
  const void* ptrs[7] = {e->walkers, e->logpost, e->lo, e->hi, e->t, e->data, e->sigma};
  for (const void* q : ptrs)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  const int64_t n = e->n_walkers, h = n / 2;
  const size_t need = ((size_t)12 * n + 2 * n + (size_t)n * e->n_times +
                       (size_t)h * (GL_FIT_DIM + 2) + n) * sizeof(double);
  int rc = grow(ctx, (void**)&ctx->d_ens, &ctx->ens_cap, need);
  if (rc) return rc;
  // exposure times (one value for every walker), stream-ordered
  double* exptime = ctx->d_ens + 12 * n + 2 * n + n * e->n_times + h * (GL_FIT_DIM + 2);
  gl_fill_kernel<<<launch_grid(n, 256), 256, 0, st>>>(exptime, n, e->exptime);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  return GL_OK;
}

int gl_ensemble_init(gl_context* ctx, const gl_ensemble* e, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_ensemble(ctx, e, st);
  if (rc) return rc;
  return ens_logpost(ctx, e, e->walkers, e->n_walkers, e->logpost, st);
}

int gl_ensemble_sweep(gl_context* ctx, const gl_ensemble* e, const double* rnd,
                      unsigned long long* accepted, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_ensemble(ctx, e, st);
  if (rc) return rc;
  if (!rnd || !is_device_ptr(rnd, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host rnd");
  if (accepted && !is_device_ptr(accepted, ctx->device))
    return fail(ctx, GL_EINVAL, "host accepted counter");
  const int64_t n = e->n_walkers, m = n / 2;
  double* prop = ctx->d_ens + 12 * n + 2 * n + n * e->n_times;
  double* z = prop + m * GL_FIT_DIM;
  double* lp_new = z + m;
  const int g = launch_grid(m, 256);
  for (int h = 0; h < 2; ++h) {
    const double* r = rnd + (size_t)h * 3 * m;   // per half: r_z, r_j, r_u (m each)
    gl_ens_propose_kernel<<<g, 256, 0, st>>>(e->walkers, m, h, r, r + m, e->a, prop, z);
    ctx->launches++;
    GL_CUDA(ctx, cudaGetLastError());
    rc = ens_logpost(ctx, e, prop, m, lp_new, st);
    if (rc) return rc;
    gl_ens_accept_kernel<<<g, 256, 0, st>>>(e->walkers, e->logpost, m, h, prop, z, lp_new,
                                            r + 2 * m, accepted);
    ctx->launches++;
    GL_CUDA(ctx, cudaGetLastError());
  }
  return GL_OK;
}

int gl_lightcurve_surrogate(gl_context* ctx, gl_mlp* mlp, const gl_params* p, const gl_times* tm,
                            double* out, const float* bound_table, double bound_limit,
                            void* stream, gl_surrogate_stats* stats) {
  NvtxRange nv("gl_lightcurve_surrogate");
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (!mlp || !p || !tm || !out || !bound_table) return fail(ctx, GL_EINVAL, "NULL argument");
  int64_t n_sets = p->n_sets, n_total = tm->n_total;
  if (n_sets < 0 || n_total < 0 || n_total >= (1LL << 31)) return fail(ctx, GL_EINVAL, "bad sizes");
  if (tm->nsuper || tm->nsuper_all < 1) return fail(ctx, GL_EINVAL, "needs a uniform nsuper_all");
  if (!tm->offsets && n_total != n_sets * tm->n_times) return fail(ctx, GL_EINVAL, "n_total");
  if (stats) memset(stats, 0, sizeof *stats);
  if (n_sets == 0 || n_total == 0) return GL_OK;
  const double* arr[15] = {p->t0, p->period, p->a_rs, p->b, p->ecc, p->omega, p->k, p->f,
                           p->eta, p->xi, p->u1, p->u2, tm->t, tm->exptime, out};
  for (const double* q : arr)
    if (!q || !is_device_ptr(q, ctx->device)) return fail(ctx, GL_EINVAL, "NULL or host array");
  if (tm->offsets && !is_device_ptr(tm->offsets, ctx->device))
    return fail(ctx, GL_EINVAL, "host offsets");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = grow(ctx, (void**)&ctx->d_sets, &ctx->sets_cap, (size_t)n_sets * sizeof(SetConst));
  if (rc) return rc;
  const int64_t items = n_total * (int64_t)tm->nsuper_all;
  if (items > ctx->sur_cap || n_total > ctx->sur_rec_cap) {
    for (void* q : {(void*)ctx->sx, (void*)ctx->sy, (void*)ctx->so, (void*)ctx->sfeat,
                    (void*)ctx->sscale, (void*)ctx->sdsph, (void*)ctx->sthat, (void*)ctx->sdef,
                    (void*)ctx->sset, (void*)ctx->scls, (void*)ctx->sfb, (void*)ctx->srj,
                    (void*)ctx->srns, (void*)ctx->srfirst})
      if (q) cudaFree(q);
    ctx->sur_cap = ctx->sur_rec_cap = 0;
    size_t fi = (size_t)items * sizeof(float), ii = (size_t)items * sizeof(int);
    size_t ri = (size_t)n_total * sizeof(int);
    bool ok = cudaMalloc(&ctx->sx, fi) == cudaSuccess && cudaMalloc(&ctx->sy, fi) == cudaSuccess &&
              cudaMalloc(&ctx->so, fi) == cudaSuccess &&
              cudaMalloc(&ctx->sfeat, 7 * fi) == cudaSuccess &&
              cudaMalloc(&ctx->sscale, fi) == cudaSuccess &&
              cudaMalloc(&ctx->sdsph, fi) == cudaSuccess &&
              cudaMalloc(&ctx->sthat, fi) == cudaSuccess &&
              cudaMalloc(&ctx->sdef, fi) == cudaSuccess && cudaMalloc(&ctx->sset, ii) == cudaSuccess &&
              cudaMalloc(&ctx->scls, ii) == cudaSuccess && cudaMalloc(&ctx->sfb, ii) == cudaSuccess &&
              cudaMalloc(&ctx->srj, ri) == cudaSuccess && cudaMalloc(&ctx->srns, ri) == cudaSuccess &&
              cudaMalloc(&ctx->srfirst, ri) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(ctx, GL_ENOMEM, "surrogate workspace of %lld items", (long long)items);
    }
    ctx->sur_cap = items;
    ctx->sur_rec_cap = n_total;
  }
  if (!ctx->scount) GL_CUDA(ctx, cudaMalloc(&ctx->scount, 3 * sizeof(unsigned long long)));
  if (!ctx->stable) GL_CUDA(ctx, cudaMalloc(&ctx->stable, kSurBins * sizeof(float)));
  GL_CUDA(ctx, cudaMemcpyAsync(ctx->stable, bound_table, kSurBins * sizeof(float), cudaMemcpyDefault, st));
  GL_CUDA(ctx, cudaMemsetAsync(ctx->scount, 0, 3 * sizeof(unsigned long long), st));
  GL_CUDA(ctx, cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned int), st));
  ParamPtrs pp;
  memset(&pp, 0, sizeof pp);
  pp.t0 = p->t0;
  pp.period = p->period;
  pp.a_rs = p->a_rs;
  pp.b = p->b;
  pp.ecc = p->ecc;
  pp.omega = p->omega;
  pp.k = p->k;
  pp.f = p->f;
  pp.eta = p->eta;
  pp.xi = p->xi;
  pp.u1 = p->u1;
  pp.u2 = p->u2;
  pp.g = p->g;
  pp.zeta = p->zeta;
  pp.exptime = tm->exptime;
  pp.nsuper_all = tm->nsuper_all;
  gl_setup_kernel<<<(int)((n_sets + 31) / 32), 128, 0, st>>>(pp, n_sets, tm->offsets, n_total,
                                                          ctx->d_sets, ctx->d_status, nullptr, 0);
  CollectArgs ca;
  memset(&ca, 0, sizeof ca);
  ca.sets = ctx->d_sets;
  ca.t = tm->t;
  ca.offsets = tm->offsets;
  ca.n_times = tm->n_times;
  ca.n_sets = n_sets;
  ca.n_total = n_total;
  ca.out = out;
  ca.tile_counter = ctx->d_counter;
  ca.tile = 256;
  ca.n_tiles = (int)((n_total + 255) / 256);
  ca.ix = ctx->sx;
  ca.iy = ctx->sy;
  ca.io = ctx->so;
  ca.iset = ctx->sset;
  ca.icls = ctx->scls;
  ca.item_cap = ctx->sur_cap;
  ca.n_items = ctx->scount;
  ca.rj = ctx->srj;
  ca.rns = ctx->srns;
  ca.rfirst = ctx->srfirst;
  ca.rec_cap = ctx->sur_rec_cap;
  ca.n_recs = ctx->scount + 1;
  ca.status = ctx->d_status;
  int grid = ctx->sms * 4;
  if (grid > ca.n_tiles) grid = ca.n_tiles;
  gl_collect_kernel<256><<<grid, 256, 0, st>>>(ca);
  ctx->launches += 2;
  GL_CUDA(ctx, cudaGetLastError());
  unsigned long long cnt[3] = {0, 0, 0};
  GL_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->scount, sizeof cnt, cudaMemcpyDeviceToHost, st));
  GL_CUDA(ctx, cudaStreamSynchronize(st));
  const int64_t n_items = (int64_t)cnt[0];
  if (n_items > 0) {
    int g2 = launch_grid(n_items, 256);
    gl_sur_features_kernel<<<g2, 256, 0, st>>>(ctx->d_sets, pp, ctx->sx, ctx->sy, ctx->so, ctx->sset,
                                               ctx->scls, ctx->scount, ctx->sfeat, ctx->sscale,
                                               ctx->sdsph);
    GL_CUDA(ctx, cudaGetLastError());
    rc = gl_mlp_forward(mlp, n_items, ctx->sfeat, ctx->sthat, stream);
    if (rc) return fail(ctx, rc, "surrogate network forward failed");
    gl_sur_combine_kernel<<<g2, 256, 0, st>>>(ctx->d_sets, p->k, ctx->sset, ctx->scls, ctx->scount,
                                              ctx->sthat, ctx->sscale, ctx->sdsph, ctx->stable,
                                              (float)bound_limit, ctx->sdef, ctx->sfb,
                                              ctx->scount + 2);
    gl_sur_fallback_kernel<<<g2, 256, 0, st>>>(ctx->d_sets, ctx->sx, ctx->sy, ctx->so, ctx->sset,
                                               ctx->scls, ctx->sfb, ctx->scount + 2, ctx->sdef);
    gl_sur_reduce_kernel<<<launch_grid((int64_t)cnt[1], 256), 256, 0, st>>>(
        ctx->srj, ctx->srns, ctx->srfirst, ctx->scount + 1, ctx->sdef, out);
    ctx->launches += 4;
    GL_CUDA(ctx, cudaGetLastError());
  }
  if (stats) {
    GL_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->scount, sizeof cnt, cudaMemcpyDeviceToHost, st));
    GL_CUDA(ctx, cudaStreamSynchronize(st));
    stats->items = (int64_t)cnt[0];
    stats->exposures = (int64_t)cnt[1];
    stats->fallback = (int64_t)cnt[2];
  }
  return GL_OK;
}

int gl_flux_sky(gl_context* ctx, int64_t n, const double* x0, const double* y0, const double* z,
                const double* k, const double* f, const double* eta, const double* xi,
                const double* u1, const double* u2, double* out, gl_precision prec,
                void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision %d", (int)prec);
  if (n == 0) return GL_OK;
  if (!x0 || !y0 || !z || !k || !f || !eta || !xi || !u1 || !u2 || !out)
    return fail(ctx, GL_EINVAL, "NULL array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  SkyPtrs sp = {x0, y0, z, k, f, eta, xi, u1, u2};
  size_t b = (size_t)n * sizeof(double);
  StageItem items[] = {{(const void**)&sp.x0, b}, {(const void**)&sp.y0, b},
                       {(const void**)&sp.z, b},  {(const void**)&sp.k, b},
                       {(const void**)&sp.f, b},  {(const void**)&sp.eta, b},
                       {(const void**)&sp.xi, b}, {(const void**)&sp.u1, b},
                       {(const void**)&sp.u2, b}};
  bool any_host = false;
  int rc = stage_inputs(ctx, items, 9, st, &any_host);
  if (rc) return rc;
  bool out_host = !is_device_ptr(out, ctx->device);
  double* d_out = out;
  if (out_host) {
    rc = grow(ctx, (void**)&ctx->d_out, &ctx->out_cap, b);
    if (rc) return rc;
    d_out = ctx->d_out;
  }
  int grid = launch_grid(n, 256);
  long pe = prof_begin(ctx, GL_KERNEL_SKY, st);
  if (prec == GL_FP64)
    gl_sky_kernel<double><<<grid, 256, 0, st>>>(sp, n, d_out, ctx->d_status);
  else
    gl_sky_kernel<float><<<grid, 256, 0, st>>>(sp, n, d_out, ctx->d_status);
  prof_end(ctx, GL_KERNEL_SKY, pe, st);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  if (out_host) GL_CUDA(ctx, cudaMemcpyAsync(out, d_out, b, cudaMemcpyDeviceToHost, st));
  if (out_host || any_host) GL_CUDA(ctx, cudaStreamSynchronize(st));
  return GL_OK;
}

int gl_flux_sky_simpson(gl_context* ctx, int64_t n, const double* x0, const double* y0,
                        const double* z, const double* k, const double* f, const double* eta,
                        const double* xi, const double* u1, const double* u2, double* out,
                        int n_intervals, gl_precision prec, void* stream) {
  if (!ctx) return GL_EINVAL;
  ctx->err[0] = 0;
  if (n < 0) return fail(ctx, GL_EINVAL, "n < 0");
  if (prec != GL_FP64 && prec != GL_FP32C) return fail(ctx, GL_EINVAL, "bad precision %d", (int)prec);
  if (n_intervals < 2 || (n_intervals & 1) || n_intervals > (1 << 24))
    return fail(ctx, GL_EINVAL, "n_intervals must be even, in [2, 2^24]");
  if (n == 0) return GL_OK;
  if (!x0 || !y0 || !z || !k || !f || !eta || !xi || !u1 || !u2 || !out)
    return fail(ctx, GL_EINVAL, "NULL array");
  GL_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  SkyPtrs sp = {x0, y0, z, k, f, eta, xi, u1, u2};
  size_t b = (size_t)n * sizeof(double);
  StageItem items[] = {{(const void**)&sp.x0, b}, {(const void**)&sp.y0, b},
                       {(const void**)&sp.z, b},  {(const void**)&sp.k, b},
                       {(const void**)&sp.f, b},  {(const void**)&sp.eta, b},
                       {(const void**)&sp.xi, b}, {(const void**)&sp.u1, b},
                       {(const void**)&sp.u2, b}};
  bool any_host = false;
  int rc = stage_inputs(ctx, items, 9, st, &any_host);
  if (rc) return rc;
  bool out_host = !is_device_ptr(out, ctx->device);
  double* d_out = out;
  if (out_host) {
    rc = grow(ctx, (void**)&ctx->d_out, &ctx->out_cap, b);
    if (rc) return rc;
    d_out = ctx->d_out;
  }
  int64_t blocks = (n + 7) / 8;   // 8 warps per block, one evaluation per warp
  if (blocks > (int64_t)ctx->sms * 64) blocks = (int64_t)ctx->sms * 64;
  long pe = prof_begin(ctx, GL_KERNEL_SIMPSON, st);
  if (prec == GL_FP64)
    gl_simpson_kernel<double><<<(int)blocks, 256, 0, st>>>(sp, n, n_intervals, d_out, ctx->d_status);
  else
    gl_simpson_kernel<float><<<(int)blocks, 256, 0, st>>>(sp, n, n_intervals, d_out, ctx->d_status);
  prof_end(ctx, GL_KERNEL_SIMPSON, pe, st);
  ctx->launches++;
  GL_CUDA(ctx, cudaGetLastError());
  if (out_host) GL_CUDA(ctx, cudaMemcpyAsync(out, d_out, b, cudaMemcpyDeviceToHost, st));
  if (out_host || any_host) GL_CUDA(ctx, cudaStreamSynchronize(st));
  return GL_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free entry
// gl_lightcurve_batch_noalloc: the same setup + light-curve kernels as
// gl_lightcurve_batch, with the per-set constants kept in a fixed device array
// instead of context workspace.  The array lives for as long as the library is
// loaded, on every device that runs the entry point.
namespace {

// The header states the array's size from this layout: keep the two in step.
static_assert(sizeof(SetConst) == 576, "gl.h documents 576-byte per-set constants");
constexpr size_t kNoallocStatusOffset = (size_t)GL_NOALLOC_MAX_SETS * sizeof(SetConst);
constexpr size_t kNoallocBytes = kNoallocStatusOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mutex;
std::vector<unsigned char*> g_noalloc_ptr;   // per device: address of g_noalloc_scratch

// Once per device, with that device current: upload the node tables and look up
// the device address of the scratch array.
int noalloc_setup(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mutex);
  if ((int)g_noalloc_ptr.size() <= device) g_noalloc_ptr.resize(device + 1, nullptr);
  if (!g_noalloc_ptr[device]) {
    if (ensure_device_tables(device) != cudaSuccess) return GL_ECUDA;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return GL_ECUDA;
    }
    g_noalloc_ptr[device] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[device];
  return GL_OK;
}

}  // namespace

extern "C" int gl_lightcurve_batch_noalloc(const gl_params* p, const gl_times* tm, double* out,
                                           gl_precision prec, void* stream) {
  if (!p || !tm) return GL_EINVAL;
  if (prec != GL_FP64 && prec != GL_FP32C) return GL_EINVAL;
  int64_t n_sets = p->n_sets;
  if (n_sets < 0 || n_sets > GL_NOALLOC_MAX_SETS) return GL_EINVAL;
  if (tm->n_total < 0 || tm->n_total >= (1LL << 31)) return GL_EINVAL;
  if (!tm->offsets && (tm->n_times < 0 || tm->n_total != n_sets * tm->n_times)) return GL_EINVAL;
  if (!tm->nsuper && tm->nsuper_all < 1) return GL_EINVAL;
  if (n_sets == 0 || tm->n_total == 0) return GL_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return GL_ECUDA;
  }
  const void* ptrs[19] = {p->t0, p->period, p->a_rs, p->b,   p->ecc,     p->omega,
                          p->k,  p->f,      p->eta,  p->xi,  p->u1,      p->u2,
                          tm->t, tm->exptime, out,   tm->offsets, tm->nsuper, p->g, p->zeta};
  for (int i = 0; i < 19; ++i) {
    if (!ptrs[i]) {
      if (i >= 15) continue;   // offsets, nsuper, g and zeta are optional
      return GL_EINVAL;
    }
    if (!is_device_ptr(ptrs[i], device)) return GL_EINVAL;   // host memory would need staging
  }
  unsigned char* scratch = nullptr;
  int rc = noalloc_setup(device, &scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  SetConst* sets = (SetConst*)scratch;
  int* status = (int*)(scratch + kNoallocStatusOffset);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return GL_ECUDA;
  ParamPtrs pp = {p->t0, p->period, p->a_rs, p->b, p->ecc, p->omega, p->k, p->f,
                  p->eta, p->xi, p->u1, p->u2, p->g, p->zeta, tm->exptime, tm->nsuper,
                  tm->nsuper_all};
  gl_setup_kernel<<<(int)((n_sets + 31) / 32), 128, 0, st>>>(pp, n_sets, tm->offsets,
                                                          tm->n_total, sets, status, nullptr, 0);
  int grid = launch_grid(tm->n_total, 256);
  if (prec == GL_FP64)
    gl_curve_kernel<double><<<grid, 256, 0, st>>>(sets, tm->t, tm->offsets, tm->n_times, n_sets,
                                                  tm->n_total, out);
  else
    gl_curve_kernel<float><<<grid, 256, 0, st>>>(sets, tm->t, tm->offsets, tm->n_times, n_sets,
                                                 tm->n_total, out);
  if (cudaGetLastError() != cudaSuccess) return GL_ECUDA;
  return GL_OK;
}
