// k_sets.cu -- active-set kernels of the localized Newton method (Section 4.3, Algorithm 1;
// Section 4.4, Algorithm 2): compaction of a bitset into an ascending cell list, boundary
// set V_B, outer halo V_dB, support/boundary flagging of an update, m-hop frontier
// expansion V_nbr^{i,m}, the expand/shrink decision and the dynamic-partition step.
//
// Sets are bitsets (bit i = cell i).  Word-parallel kernels give one 32-bit word to a
// thread and write whole words (no atomics, coalesced); scatter kernels (halo, frontier)
// use atomicOr, which is idempotent, so every set is independent of thread order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lns_internal.cuh"

namespace lns {

namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ bool bit(const uint32_t* s, int i) { return (s[i >> 5] >> (i & 31)) & 1u; }

__device__ __forceinline__ uint32_t valid_mask(int w, int n) {
  int rem = n - (w << 5);
  return rem >= 32 ? 0xffffffffu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
}

// Append `value` to list when pred holds; one atomicAdd per warp.
__device__ __forceinline__ void warp_append(int* counter, int* list, bool pred, int value) {
  unsigned act = __activemask();
  unsigned m = __ballot_sync(act, pred);
  if (!pred) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(m, base, leader);
  list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// Set bit i of a bitset when pred holds: the lanes of a warp that set bits of the same word are
// grouped and one of them applies their bits with one atomicOr (the rows of a warp are ascending
// cells, so a warp touches a few words instead of issuing 32 atomics on each).
__device__ __forceinline__ void warp_set_bit(uint32_t* words, bool pred, int i) {
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, pred);
  if (!pred) return;
  const int w = i >> 5;
  const unsigned grp = __match_any_sync(m, w);
  const unsigned bits = __reduce_or_sync(grp, 1u << (i & 31));
  if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicOr(&words[w], bits);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------------------
// Compaction of a bitset: ascending list of set cells and the inverse map.
// Pass 1: popcount per block of kBlk words.  Pass 2: each block sums the counts of the
// blocks before it, scans its words and writes list[] and inv[].  Small bitsets take pass 2 alone,
// each block counting the earlier words itself.
// ---------------------------------------------------------------------------------------
__global__ void k_compact_count(const uint32_t* __restrict__ bits, int W, int* __restrict__ blk_sums) {
  int w = blockIdx.x * kBlk + threadIdx.x;
  int c = (w < W) ? __popc(bits[w]) : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ int ws[kBlk / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < kBlk / 32; k++) s += ws[k];
    blk_sums[blockIdx.x] = s;
  }
}

// FUSED: one pass for small bitsets (kFuseWords words at most): each block counts the set bits of
// all the words before its own itself (at most kFuseWords / kBlk loads a thread), so the counting
// pass and its launch go away.
constexpr int kFuseWords = 8192;

template <bool FUSED>
__global__ void k_compact_write(const uint32_t* __restrict__ bits, int W, const int* __restrict__ blk_sums,
                                int* __restrict__ list, int* __restrict__ inv, int* __restrict__ count_out) {
  __shared__ int ws[kBlk / 32];
  __shared__ int s_off;
  // offset of this block = sum of the counts of earlier blocks (of the words before it)
  int part = 0;
  if (FUSED) {
    for (int v = threadIdx.x; v < (int)blockIdx.x * kBlk; v += kBlk) part += __popc(bits[v]);
  } else {
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kBlk) part += blk_sums[b];
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < kBlk / 32; k++) s += ws[k];
    s_off = s;
  }
  __syncthreads();
  int w = blockIdx.x * kBlk + threadIdx.x;
  uint32_t word = (w < W) ? bits[w] : 0u;
  int c = __popc(word);
  // block exclusive scan of c
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = c;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  int wpre = 0;
  for (int k = 0; k < warp; k++) wpre += ws[k];
  int pos = s_off + wpre + inc - c;
  while (word) {
    int b = __ffs(word) - 1;
    word &= word - 1u;
    int cell = (w << 5) + b;
    list[pos] = cell;
    if (inv) inv[cell] = pos;
    pos++;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kBlk - 1) *count_out = pos;
}

// V_B: cells of the set with at least one neighbour outside it.  One word per thread.
__global__ void k_boundary(const int* __restrict__ row_ptr, const int* __restrict__ nbr,
                           const uint32_t* __restrict__ set, int W, uint32_t* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  uint32_t word = set[w], res = 0u;
  while (word) {
    int b = __ffs(word) - 1;
    word &= word - 1u;
    int i = (w << 5) + b;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++)
      if (!bit(set, nbr[e])) {
        res |= 1u << b;
        break;
      }
  }
  out[w] = res;
}

// V_dB: cells outside the set with a neighbour inside it (scatter from the set's list).
__global__ void k_outer_halo(const int* __restrict__ row_ptr, const int* __restrict__ nbr,
                             const uint32_t* __restrict__ set, const int* __restrict__ list,
                             const int* __restrict__ count, uint32_t* __restrict__ out) {
  int nl = *count;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nl; k += gridDim.x * blockDim.x) {
    int i = list[k];
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      int j = nbr[e];
      if (!bit(set, j)) atomicOr(&out[j >> 5], 1u << (j & 31));
    }
  }
}

// Flag the update of the active rows.  With x != nullptr the update comes from the Krylov
// solution (scaled unknowns): du = (x0 / p_scale, chop(x1)), stored in dp/dsw and added to
// the state when `apply`.  Otherwise dp/dsw already hold the caller's update.
//   support S (bits), boundary cells with |du| >= eps -> frontier list 0 and reach bits,
//   max |dp|, max |dsw|, Algorithm 2 stamps.
__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) r = fmax(r, sh[k]);
  __syncthreads();
  return r;
}

template <typename T>
__global__ void k_flag(Dev d, const uint32_t* __restrict__ vb, int apply, int record_stamp, int solve_id,
                       double eps_p, double eps_sw, double p_scale, double sat_chop, const T* __restrict__ x,
                       double fail_rtol) {
  __shared__ double sh[32];
  const double inv_p_scale = 1.0 / p_scale;  // once per thread, outside the row loop
  int nA = d.ctr->n_active;
  // A failed Krylov solve (breakdown, a barrier wait that gave up, or a stop far from the
  // tolerance) changes nothing: no update, no support, no frontier, so the iteration can be
  // redone from the same state and set.
  if (x && apply) {
    const int st = d.ctr->krylov_status;
    if (st == 2 || st == 3 || (st == 1 && !(d.ctr->krylov_relres <= fail_rtol))) {
      if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr->solve_failed = 1;
      return;
    }
  }
  double mdp = 0.0, mds = 0.0;
  int any_s = 0, any_e = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nA; k += gridDim.x * blockDim.x) {
    int i = d.act[k];
    double dp, dsw;
    if (x) {
      dp = (double)x[2 * k] * inv_p_scale;
      dsw = (double)x[2 * k + 1];
      if (sat_chop > 0.0) dsw = fmin(fmax(dsw, -sat_chop), sat_chop);
      d.dp[i] = dp;
      d.dsw[i] = dsw;
      if (apply) {
        d.p[i] += dp;
        d.sw[i] += dsw;
      }
    } else {
      dp = d.dp[i];
      dsw = d.dsw[i];
    }
    bool big = fabs(dp) >= eps_p || (eps_sw > 0.0 && fabs(dsw) >= eps_sw);
    mdp = fmax(mdp, fabs(dp));
    mds = fmax(mds, fabs(dsw));
    bool edge = big && vb != nullptr && bit(vb, i);
    if (big) {
      if (record_stamp) d.stamp[i] = solve_id;
      any_s = 1;
    }
    warp_set_bit(d.supp, big, i);
    warp_set_bit(d.reach, edge, i);
    any_e |= edge;
    warp_append(&d.ctr->n_frontier[0], d.fr0, edge, i);
  }
  // blocks with no rows (small systems leave most of the grid idle) skip the reductions and the
  // counter atomics, which all land on one line
  if ((int)(blockIdx.x * blockDim.x) >= nA) return;
  any_s = __syncthreads_or(any_s);
  any_e = __syncthreads_or(any_e);
  mdp = block_max(mdp, sh);
  mds = block_max(mds, sh);
  if (threadIdx.x == 0) {
    if (mdp > 0.0) atomic_max_nonneg(&d.ctr->max_dp_bits, mdp);
    if (mds > 0.0) atomic_max_nonneg(&d.ctr->max_dsw_bits, mds);
    if (any_s) atomicOr(&d.ctr->any_s, 1);
    if (any_e) atomicOr(&d.ctr->any_e, 1);
  }
}

// One hop of the m-layer expansion: every neighbour of the frontier joins `reach`; newly
// reached cells form the next frontier.
__global__ void k_dilate_round(const int* __restrict__ row_ptr, const int* __restrict__ nbr,
                               const int* __restrict__ fin, const int* __restrict__ cin, int* __restrict__ fout,
                               int* __restrict__ cout, uint32_t* __restrict__ reach) {
  int nf = *cin;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
    int i = fin[k];
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      int j = nbr[e];
      uint32_t m = 1u << (j & 31);
      uint32_t old = atomicOr(&reach[j >> 5], m);
      bool fresh = !(old & m);
      if (fresh) {
        int pos = atomicAdd(cout, 1);
        fout[pos] = j;
      }
    }
  }
}

__global__ void k_seed(const int* __restrict__ list, int count, uint32_t* __restrict__ reach,
                       int* __restrict__ fr, int* __restrict__ cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    int i = list[k];
    atomicOr(&reach[i >> 5], 1u << (i & 31));
    fr[k] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = count;
}

// Algorithm 1, lines 8-20: expand (V_A |= reach) if a boundary cell moved, else shrink to
// the support (an empty support before convergence keeps V_A).  Also accumulates the
// union of the solved sets of the timestep.
__global__ void k_alg1_combine(Dev d, double tol_dp, double tol_cnv, int converged_override) {
  IterCounters* c = d.ctr;
  double maxdp = __longlong_as_double((long long)c->max_dp_bits);
  double cnv = __longlong_as_double((long long)c->cnv_bits);
  int conv = converged_override >= 0 ? converged_override : (maxdp < tol_dp && cnv < tol_cnv);
  int any_e = c->any_e, any_s = c->any_s;
  const int failed = c->solve_failed;  // V_A stays as it was for a redo of the iteration
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0) {
    c->converged = failed ? 0 : conv;
    c->is_expand = failed ? 0 : (any_e ? 1 : 0);
  }
  if (w >= d.W || failed) return;
  uint32_t va = d.va[w];
  d.uni[w] |= va;
  if (any_e)
    va = va | d.reach[w] | d.always[w];
  else if (any_s || conv)
    va = d.supp[w] | d.always[w];
  d.va[w] = va;
}

// Algorithm 2, lines 8-15: next subdomain = reached cells not yet in V_T; V_T |= reached.
__global__ void k_dd_combine(Dev d, const uint32_t* __restrict__ reach, uint32_t* __restrict__ vt,
                             uint32_t* __restrict__ va_next) {
  int any_e = d.ctr->any_e;
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= d.W) return;
  uint32_t r = any_e ? reach[w] : 0u;
  uint32_t nxt = r & ~vt[w];
  va_next[w] = nxt;
  vt[w] |= r;
  if (nxt) atomicOr(&d.ctr->any_new, 1);
}

__global__ void k_words(int W, int n, int op, uint32_t* __restrict__ out, const uint32_t* __restrict__ a,
                        const uint32_t* __restrict__ b) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  uint32_t r;
  switch (op) {
    case kCopy: r = a[w]; break;
    case kOr: r = a[w] | b[w]; break;
    case kAnd: r = a[w] & b[w]; break;
    case kAndNot: r = a[w] & ~b[w]; break;
    default: r = valid_mask(w, n); break;  // kAll
  }
  out[w] = r;
}

// Support of the timestep's update (next step's initial set): cells with |p - p^n| >= eps.
// Only cells of the step's union can have changed; others have a zero update.
__global__ void k_step_support(Dev d, double eps_p, double eps_sw) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= d.W) return;
  uint32_t u = d.uni[w], res = 0u;
  bool zero_big = (0.0 >= eps_p) || (eps_sw > 0.0 && 0.0 >= eps_sw);
  uint32_t valid = valid_mask(w, d.n);
  for (int b = 0; b < 32; b++) {
    if (!((valid >> b) & 1u)) break;
    bool big;
    if ((u >> b) & 1u) {
      int i = (w << 5) + b;
      double dp = d.p[i] - d.pn[i], dsw = d.sw[i] - d.swn[i];
      big = fabs(dp) >= eps_p || (eps_sw > 0.0 && fabs(dsw) >= eps_sw);
    } else {
      big = zero_big;
    }
    if (big) res |= 1u << b;
  }
  d.prev[w] = res;
}

// Algorithm 2, line 27: did a cell of V_dB^k receive a non-negligible update after solve `since`?
__global__ void k_halo_check(Dev d, const uint32_t* __restrict__ vdb, int since) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= d.W) return;
  uint32_t word = vdb[w];
  while (word) {
    int b = __ffs(word) - 1;
    word &= word - 1u;
    if (d.stamp[(w << 5) + b] > since) {
      atomicOr(&d.ctr->halo_flag, 1);
      return;
    }
  }
}

inline int words_grid(int W) { return (W + kBlk - 1) / kBlk; }

}  // namespace

// grid of the per-iteration list kernels (update/flag, frontier expansion, halo): blocks per SM x SMs
static int set_grid(const LaunchCfg& c) { return (c.set_mult >= 1 && c.set_mult <= 16 ? c.set_mult : 4) * c.sms; }

cudaError_t launch_compact(const Dev& d, const uint32_t* bits, int* list, int* inv, int* count_out, LaunchCfg c) {
  int nb = words_grid(d.W);
  if (nb == 0) return cudaMemsetAsync(count_out, 0, sizeof(int), c.stream);
  if (d.W <= kFuseWords) {
    count_launches(1);
    k_compact_write<true><<<nb, kBlk, 0, c.stream>>>(bits, d.W, nullptr, list, inv, count_out);
    return cudaGetLastError();
  }
  count_launches(1);
  k_compact_count<<<nb, kBlk, 0, c.stream>>>(bits, d.W, d.blk_sums);
  count_launches(1);
  k_compact_write<false><<<nb, kBlk, 0, c.stream>>>(bits, d.W, d.blk_sums, list, inv, count_out);
  return cudaGetLastError();
}

cudaError_t launch_boundary(const Dev& d, const uint32_t* set, uint32_t* out, LaunchCfg c) {
  if (d.W == 0) return cudaSuccess;
  count_launches(1);
  k_boundary<<<words_grid(d.W), kBlk, 0, c.stream>>>(d.row_ptr, d.nbr, set, d.W, out);
  return cudaGetLastError();
}

cudaError_t launch_outer_halo(const Dev& d, const uint32_t* set, const int* list, const int* count, uint32_t* out,
                              LaunchCfg c) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t) * (size_t)d.W, c.stream);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_outer_halo<<<set_grid(c), kBlk, 0, c.stream>>>(d.row_ptr, d.nbr, set, list, count, out);
  return cudaGetLastError();
}

cudaError_t launch_flag(const Dev& d, const uint32_t* vb, int apply, int record_stamp, int solve_id, double eps_p,
                        double eps_sw, double p_scale, double sat_chop, int fp32, const void* x, double fail_rtol,
                        LaunchCfg c) {
  count_launches(1);
  if (fp32)
    k_flag<float><<<set_grid(c), kBlk, 0, c.stream>>>(d, vb, apply, record_stamp, solve_id, eps_p, eps_sw, p_scale,
                                                    sat_chop, (const float*)x, fail_rtol);
  else
    k_flag<double><<<set_grid(c), kBlk, 0, c.stream>>>(d, vb, apply, record_stamp, solve_id, eps_p, eps_sw, p_scale,
                                                     sat_chop, (const double*)x, fail_rtol);
  return cudaGetLastError();
}

// m rounds of frontier expansion starting from frontier list 0 (already seeded in reach).
cudaError_t launch_dilate(const Dev& d, uint32_t* reach, int layers, LaunchCfg c) {
  for (int h = 0; h < layers; h++) {
    const int* fin = (h & 1) ? d.fr1 : d.fr0;
    int* fout = (h & 1) ? d.fr0 : d.fr1;
    const int* cin = &d.ctr->n_frontier[h & 1];
    int* cout = &d.ctr->n_frontier[(h + 1) & 1];
    cudaError_t e = cudaMemsetAsync(cout, 0, sizeof(int), c.stream);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_dilate_round<<<set_grid(c), kBlk, 0, c.stream>>>(d.row_ptr, d.nbr, fin, cin, fout, cout, reach);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_seed_frontier(const Dev& d, const int* list, int count_host, uint32_t* reach, LaunchCfg c) {
  count_launches(1);
  k_seed<<<set_grid(c), kBlk, 0, c.stream>>>(list, count_host, reach, d.fr0, &d.ctr->n_frontier[0]);
  return cudaGetLastError();
}

cudaError_t launch_alg1_combine(const Dev& d, double tol_dp, double tol_cnv, int converged_override, LaunchCfg c) {
  count_launches(1);
  k_alg1_combine<<<words_grid(d.W > 0 ? d.W : 1), kBlk, 0, c.stream>>>(d, tol_dp, tol_cnv, converged_override);
  return cudaGetLastError();
}

cudaError_t launch_dd_combine(const Dev& d, const uint32_t* reach, uint32_t* vt, uint32_t* va_next, LaunchCfg c) {
  if (d.W == 0) return cudaSuccess;
  count_launches(1);
  k_dd_combine<<<words_grid(d.W), kBlk, 0, c.stream>>>(d, reach, vt, va_next);
  return cudaGetLastError();
}

cudaError_t launch_words_op(const Dev& d, int op, uint32_t* out, const uint32_t* a, const uint32_t* b, LaunchCfg c) {
  if (d.W == 0) return cudaSuccess;
  count_launches(1);
  k_words<<<words_grid(d.W), kBlk, 0, c.stream>>>(d.W, d.n, op, out, a, b);
  return cudaGetLastError();
}

cudaError_t launch_step_support(const Dev& d, double eps_p, double eps_sw, LaunchCfg c) {
  if (d.W == 0) return cudaSuccess;
  count_launches(1);
  k_step_support<<<words_grid(d.W), kBlk, 0, c.stream>>>(d, eps_p, eps_sw);
  return cudaGetLastError();
}

cudaError_t launch_halo_check(const Dev& d, const uint32_t* vdb, int since, LaunchCfg c) {
  cudaError_t e = cudaMemsetAsync(&d.ctr->halo_flag, 0, sizeof(int), c.stream);
  if (e != cudaSuccess) return e;
  if (d.W == 0) return cudaSuccess;
  count_launches(1);
  k_halo_check<<<words_grid(d.W), kBlk, 0, c.stream>>>(d, vdb, since);
  return cudaGetLastError();
}

}  // namespace lns
