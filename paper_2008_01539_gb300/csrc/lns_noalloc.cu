// lns_noalloc.cu -- the active-set update of lns_active_set for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: their device memory belongs to a host framework's pool
// or to a fixed budget handed out in advance, or they run where a device allocation (which can
// synchronize the whole device) would stall other work.  lns_model_create allocates, so such a
// caller cannot hold a model.  lns_active_set_noalloc gives them the same set update on arrays
// they already own: every input and output is the caller's device memory, and the working
// storage (frontier lists, support and boundary bitsets, counters) is the file-scope array
// g_noalloc_scratch below, which every GPU that loads the library keeps until the process exits.
//
// The scratch is shared by all calls: a call clears what it needs cleared, and two calls that
// overlap on the GPU (different streams, or different host threads on one device) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "lns_internal.cuh"

namespace {

constexpr int kMaxCells = LNS_NOALLOC_MAX_CELLS;
constexpr int kMaxWords = (kMaxCells + 31) / 32;
constexpr int kBlk = 256;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffFr0 = 0;
constexpr size_t kOffFr1 = kOffFr0 + sizeof(int) * (size_t)kMaxCells;
constexpr size_t kOffVbOld = kOffFr1 + sizeof(int) * (size_t)kMaxCells;
constexpr size_t kOffSupp = kOffVbOld + sizeof(uint32_t) * (size_t)kMaxWords;
constexpr size_t kOffReach = kOffSupp + sizeof(uint32_t) * (size_t)kMaxWords;
constexpr size_t kOffCtr = kOffReach + sizeof(uint32_t) * (size_t)kMaxWords;
constexpr size_t kCtrInts = 64;  // [0..1] frontier counts, [2] any boundary update, [3] any support
constexpr size_t kScratchBytes = kOffCtr + sizeof(int) * kCtrInts;
static_assert(kOffVbOld % 256 == 0 && kOffSupp % 256 == 0 && kOffReach % 256 == 0 && kOffCtr % 256 == 0,
              "scratch regions must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
  int *fr0, *fr1, *ctr;
  uint32_t *vb_old, *supp, *reach;
};

// Host-side device address of g_noalloc_scratch for each device (looked up once per device, with
// that device current).  The host symbol itself is not a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_base[kMaxDevices] = {nullptr};

__device__ __forceinline__ bool bit(const uint32_t* s, int i) { return (s[i >> 5] >> (i & 31)) & 1u; }

__device__ __forceinline__ uint32_t valid_mask(int w, int n) {
  const int rem = n - (w << 5);
  return rem >= 32 ? 0xffffffffu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
}

// V_B of a set: members with at least one neighbour outside it (one word per thread).
__global__ void k_na_boundary(const int* __restrict__ row_ptr, const int* __restrict__ nbr,
                              const uint32_t* __restrict__ set, int W, int n, uint32_t* __restrict__ out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  uint32_t word = set[w] & valid_mask(w, n), res = 0u;
  while (word) {
    const int b = __ffs(word) - 1;
    word &= word - 1u;
    const int i = (w << 5) + b;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++)
      if (!bit(set, nbr[e])) {
        res |= 1u << b;
        break;
      }
  }
  out[w] = res;
}

// Support of the update over V_A and its boundary cells with a non-negligible update (seeds
// of the expansion), one word per thread.
__global__ void k_na_flag(const uint32_t* __restrict__ va, const double* __restrict__ dp,
                          const double* __restrict__ dsw, double eps_p, double eps_sw, int W, int n, Scratch s) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  uint32_t word = va[w] & valid_mask(w, n), supp = 0u, edge = 0u;
  const uint32_t vbw = s.vb_old[w];
  while (word) {
    const int b = __ffs(word) - 1;
    word &= word - 1u;
    const int i = (w << 5) + b;
    const double dsi = dsw ? dsw[i] : 0.0;
    const bool big = fabs(dp[i]) >= eps_p || (eps_sw > 0.0 && fabs(dsi) >= eps_sw);
    if (big) {
      supp |= 1u << b;
      if ((vbw >> b) & 1u) {
        edge |= 1u << b;
        const int pos = atomicAdd(&s.ctr[0], 1);
        s.fr0[pos] = i;
      }
    }
  }
  s.supp[w] = supp;
  s.reach[w] = edge;
  if (supp) atomicOr(&s.ctr[3], 1);
  if (edge) atomicOr(&s.ctr[2], 1);
}

// One hop of V_nbr^{i,m}: neighbours of the frontier join `reach`; new cells form the next frontier.
__global__ void k_na_dilate(const int* __restrict__ row_ptr, const int* __restrict__ nbr, const int* __restrict__ fin,
                            const int* __restrict__ cin, int* __restrict__ fout, int* __restrict__ cout,
                            uint32_t* __restrict__ reach) {
  const int nf = *cin;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
    const int i = fin[k];
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      const int j = nbr[e];
      const uint32_t m = 1u << (j & 31);
      if (!(atomicOr(&reach[j >> 5], m) & m)) fout[atomicAdd(cout, 1)] = j;
    }
  }
}

// Expand (V_A |= reach) or shrink to the support (an empty support before convergence keeps V_A).
__global__ void k_na_combine(uint32_t* __restrict__ va, const uint32_t* __restrict__ always, int W, int n,
                             int converged, Scratch s) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int any_e = s.ctr[2], any_s = s.ctr[3];
  const uint32_t valid = valid_mask(w, n);
  const uint32_t alw = always ? (always[w] & valid) : 0u;
  uint32_t v = va[w] & valid;
  if (any_e)
    v = v | s.reach[w] | alw;
  else if (any_s || converged)
    v = s.supp[w] | alw;
  va[w] = v;
}

lns_status fail(lns_status s, const std::string& m) {
  lns::set_last_error(m.c_str());
  return s;
}

// Device address of the scratch array on the current device (once per device).
lns_status scratch_for_current_device(Scratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LNS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LNS_EINVAL, "device ordinal out of range");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(LNS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_base[dev] = p;
    }
    base = g_base[dev];
  }
  unsigned char* b = (unsigned char*)base;
  out->fr0 = (int*)(b + kOffFr0);
  out->fr1 = (int*)(b + kOffFr1);
  out->vb_old = (uint32_t*)(b + kOffVbOld);
  out->supp = (uint32_t*)(b + kOffSupp);
  out->reach = (uint32_t*)(b + kOffReach);
  out->ctr = (int*)(b + kOffCtr);
  return LNS_OK;
}

}  // namespace

extern "C" lns_status lns_active_set_noalloc(int32_t n_cells, const int32_t* row_ptr, const int32_t* nbr,
                                             const uint32_t* always_bits, const double* dp, const double* dsw,
                                             double eps_p, double eps_sw, int32_t m_layers, int32_t converged,
                                             uint32_t* va_bits, uint32_t* vb_bits, int32_t* is_expand,
                                             void* cuda_stream) {
  if (n_cells < 0 || n_cells > kMaxCells)
    return fail(LNS_EINVAL, "n_cells must be in [0, " + std::to_string(kMaxCells) +
                                "] for lns_active_set_noalloc (its scratch array is sized for that many cells)");
  if (m_layers < 0 || m_layers > LNS_NOALLOC_MAX_LAYERS)
    return fail(LNS_EINVAL, "m_layers must be in [0, " + std::to_string(LNS_NOALLOC_MAX_LAYERS) + "]");
  if (!(eps_p >= 0.0)) return fail(LNS_EINVAL, "eps_p must be >= 0");
  if (!is_expand) return fail(LNS_EINVAL, "is_expand must be non-NULL");
  if (n_cells == 0) {
    *is_expand = 0;
    return LNS_OK;
  }
  if (!row_ptr || !nbr || !dp || !va_bits || !vb_bits)
    return fail(LNS_EINVAL, "row_ptr, nbr, dp, va_bits and vb_bits must be device pointers (non-NULL)");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  {  // the call waits for its stream, which a stream capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(stream, &cap);
    if (ce != cudaSuccess) return fail(LNS_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(LNS_EINVAL, "lns_active_set_noalloc waits for its stream and cannot be called during a capture");
  }
  Scratch s;
  lns_status st = scratch_for_current_device(&s);
  if (st != LNS_OK) return st;
  const int W = (n_cells + 31) / 32;
  const int grid = (W + kBlk - 1) / kBlk;
  cudaError_t e = cudaMemsetAsync(s.ctr, 0, sizeof(int) * kCtrInts, stream);
  if (e == cudaSuccess) {
    k_na_boundary<<<grid, kBlk, 0, stream>>>(row_ptr, nbr, va_bits, W, n_cells, s.vb_old);
    k_na_flag<<<grid, kBlk, 0, stream>>>(va_bits, dp, dsw, eps_p, eps_sw, W, n_cells, s);
    lns::count_launches(2);
    for (int h = 0; h < m_layers && e == cudaSuccess; h++) {
      int* cin = &s.ctr[h & 1];
      int* cout = &s.ctr[(h + 1) & 1];
      e = cudaMemsetAsync(cout, 0, sizeof(int), stream);
      if (e != cudaSuccess) break;
      const int dgrid = std::min(1024, (n_cells + kBlk - 1) / kBlk);
      k_na_dilate<<<dgrid, kBlk, 0, stream>>>(row_ptr, nbr, (h & 1) ? s.fr1 : s.fr0, cin, (h & 1) ? s.fr0 : s.fr1,
                                              cout, s.reach);
      lns::count_launches(1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    k_na_combine<<<grid, kBlk, 0, stream>>>(va_bits, always_bits, W, n_cells, converged ? 1 : 0, s);
    k_na_boundary<<<grid, kBlk, 0, stream>>>(row_ptr, nbr, va_bits, W, n_cells, vb_bits);
    lns::count_launches(2);
    e = cudaGetLastError();
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, &s.ctr[2], sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(LNS_ECUDA, std::string("lns_active_set_noalloc: ") + cudaGetErrorString(e));
  *is_expand = flag ? 1 : 0;
  return LNS_OK;
}
