// pj_pair_bounds_static: the per-pair LoD bounds of pj_pair_bounds without
// any device allocation.  Its scratch (pair set-up data, per-pair bound
// words, tile counts and offsets, the tile list, counters) lives in one
// file-scope __device__ array of fixed size that every GPU which loads the
// library holds until the process exits.  Inputs and outputs are caller
// device buffers.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side shadow); the device address is obtained once per device
// with cudaGetSymbolAddress while that device is current, cached, and passed
// to the kernels.  All calls share the array and find the previous call's
// contents in it: everything that must start at zero is cleared here, and
// calls that overlap on the GPU (two streams, or two host threads) race on
// the same bytes.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace pj {

namespace {

constexpr int64_t MAXP = PJ_STATIC_MAX_PAIRS;
constexpr int64_t MAXT = PJ_STATIC_MAX_TILES;
constexpr int64_t MAXQ = 65536;   // queued straddling facet pairs

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the regions inside the scratch array
constexpr size_t OFF_ORIGIN = 0;
constexpr size_t OFF_THR = OFF_ORIGIN + align256(MAXP * 16);
constexpr size_t OFF_BOXLB = OFF_THR + align256(MAXP * 4);
constexpr size_t OFF_ANCUB = OFF_BOXLB + align256(MAXP * 8);
constexpr size_t OFF_DLO = OFF_ANCUB + align256(MAXP * 8);
constexpr size_t OFF_DHI = OFF_DLO + align256(MAXP * 8);
constexpr size_t OFF_D = OFF_DHI + align256(MAXP * 8);
constexpr size_t OFF_STATUS = OFF_D + align256(MAXP * 8);
constexpr size_t OFF_LOD0 = OFF_STATUS + align256(MAXP);
constexpr size_t OFF_EXACT = OFF_LOD0 + align256(MAXP);
constexpr size_t OFF_LB = OFF_EXACT + align256(MAXP);
constexpr size_t OFF_UB = OFF_LB + align256(MAXP * 8);
constexpr size_t OFF_MID = OFF_UB + align256(MAXP * 8);
constexpr size_t OFF_TILES = OFF_MID + align256(MAXP * 8);
constexpr size_t OFF_UCOUNT = OFF_TILES + align256(MAXT * sizeof(Tile));
constexpr size_t OFF_QUEUE = OFF_UCOUNT + 256;
constexpr size_t OFF_COUNTERS = OFF_QUEUE + align256(MAXQ * sizeof(int4));
constexpr size_t OFF_ERR = OFF_COUNTERS + 256;
constexpr size_t SCRATCH_BYTES = OFF_ERR + 256;

}  // namespace

// The scratch itself: about 2.4 MB per device.
static __device__ __align__(256) unsigned char g_bounds_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_mu;
void* g_addr[64] = {};   // device address of g_bounds_scratch, per device ordinal

// pair ids outside [0, nR) x [0, nS) are reported instead of read through
__global__ void k_check_ids(int64_t n, const int32_t* pr, const int32_t* ps, int nR, int nS) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int* err = reinterpret_cast<int*>(g_bounds_scratch + OFF_ERR);
  if (pr[p] < 0 || pr[p] >= nR || ps[p] < 0 || ps[p] >= nS) atomicOr(err, ERR_BOUNDS);
}

__global__ void k_bits_out(int64_t n, int fp64, const void* lb, const void* ub, double* lo, double* hi) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (fp64) {
    lo[p] = __longlong_as_double(((const long long*)lb)[p]);
    hi[p] = __longlong_as_double(((const long long*)ub)[p]);
  } else {
    lo[p] = (double)__uint_as_float(((const unsigned*)lb)[p]);
    hi[p] = (double)__uint_as_float(((const unsigned*)ub)[p]);
  }
}

// Device address of the scratch for the current device (set-up on first use).
unsigned char* scratch_for(int device) {
  if (device < 0 || device >= 64) throw ApiError{PJ_EINVAL, "device ordinal above 63"};
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_bounds_scratch);
    if (e != cudaSuccess) throw CudaError{e, "cudaGetSymbolAddress(g_bounds_scratch)"};
    g_addr[device] = p;
  }
  return static_cast<unsigned char*>(g_addr[device]);
}

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" pj_status pj_pair_bounds_static(pj_ctx* ctx, const pj_set* R, const pj_set* S, const int32_t* pr,
                                           const int32_t* ps, int64_t n, int lod, pj_precision prec, double* lb,
                                           double* ub, void* cuda_stream) {
  if (!ctx || !R || !S || n < 0 || (n > 0 && (!pr || !ps || !lb || !ub))) {
    if (ctx) ctx->last_error = "bad pair_bounds_static arguments";
    return PJ_EINVAL;
  }
  if (R->streamed || S->streamed || lod < 0 || lod >= R->L || lod >= S->L) {
    ctx->last_error = "pair_bounds_static: streamed set or lod out of range";
    return PJ_EINVAL;
  }
  if (n > MAXP) {
    ctx->last_error = "pair_bounds_static: n = " + std::to_string(n) + " exceeds PJ_STATIC_MAX_PAIRS (" +
                      std::to_string(MAXP) + ")";
    return PJ_EINVAL;
  }
  // worst-case unit count: every block pair of the largest objects at this LoD
  const int64_t br = (R->lod[lod].maxF + BLK - 1) / BLK, bs = (S->lod[lod].maxF + BLK - 1) / BLK;
  if (n * br * bs > MAXT) {
    ctx->last_error = "pair_bounds_static: up to " + std::to_string(n * br * bs) +
                      " units needed, above PJ_STATIC_MAX_TILES (" + std::to_string(MAXT) + ")";
    return PJ_EINVAL;
  }
  if (n == 0) return PJ_OK;
  try {
    PJ_CK(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    unsigned char* base = scratch_for(ctx->device);
    int* err = reinterpret_cast<int*>(base + OFF_ERR);
    // clear what must start at zero: error word and counters
    PJ_CK(cudaMemsetAsync(base + OFF_COUNTERS, 0, 512, st));
    int th = 256;
    k_check_ids<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, pr, ps, R->n, S->n);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    int herr = 0;
    PJ_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
    if (herr & ERR_BOUNDS) {
      ctx->last_error = "pair_bounds_static: pair id out of range";
      return PJ_EBOUNDS;
    }
    PairBufs b;
    b.pr = pr;
    b.ps = ps;
    b.origin = reinterpret_cast<float4*>(base + OFF_ORIGIN);
    b.thr = reinterpret_cast<float*>(base + OFF_THR);
    b.box_lb = reinterpret_cast<double*>(base + OFF_BOXLB);
    b.anc_ub = reinterpret_cast<double*>(base + OFF_ANCUB);
    b.status = base + OFF_STATUS;
    b.lod0 = base + OFF_LOD0;
    b.exact = base + OFF_EXACT;
    b.dlo = reinterpret_cast<double*>(base + OFF_DLO);
    b.dhi = reinterpret_cast<double*>(base + OFF_DHI);
    b.d = reinterpret_cast<double*>(base + OFF_D);
    b.lb = base + OFF_LB;
    b.ub = base + OFF_UB;
    b.mid = base + OFF_MID;
    b.tiles = reinterpret_cast<Tile*>(base + OFF_TILES);
    b.counters = reinterpret_cast<unsigned long long*>(base + OFF_COUNTERS);
    b.queue = reinterpret_cast<int4*>(base + OFF_QUEUE);
    b.flag = nullptr;
    b.qcap = (unsigned)MAXQ;
    b.tiles_cap = MAXT;
    StepSpec sp;
    sp.lodR = lod;
    sp.lodS = lod;
    sp.full = (lod == R->L - 1) && (lod == S->L - 1);
    sp.fp64 = prec == PJ_PREC_FP64;
    sp.cull = false;
    sp.want = UNDECIDED;
    sp.step = 0;
    sp.exact_cross = true;
    b.ucount = reinterpret_cast<int64_t*>(base + OFF_UCOUNT);
    b.err = err;
    setup_pairs_bufs(ctx, R, S, n, b, st);
    init_bounds_bufs(ctx, n, sp, b, st);
    const UnitCount total = build_tiles_bufs(ctx, R, S, n, sp, b, MAXT, st);
    run_refine_bufs(ctx, R, S, total, sp, b, err, st);
    k_bits_out<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(n, sp.fp64 ? 1 : 0, b.lb, b.ub, lb, ub);
    PJ_CK(cudaGetLastError());
    PJ_COUNT_LAUNCH;
    PJ_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PJ_CK(cudaStreamSynchronize(st));
    if (herr & ERR_MBAR_TIMEOUT) {
      ctx->last_error = "a device wait hit its limit";
      return PJ_ETIMEOUT;
    }
    return PJ_OK;
  } catch (const CudaError& e) {
    ctx->last_error = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    return PJ_ECUDA;
  } catch (const ApiError& e) {
    ctx->last_error = e.msg;
    return e.st;
  }
}
