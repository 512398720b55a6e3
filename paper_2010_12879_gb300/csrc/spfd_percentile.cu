// Step 6 of the pipeline (Sec. II-A, step 6; Sec. III-E): the 99th
// percentile of the voxel-averaged |E|, per tissue and over the whole body.
//
// The p-quantile of n values is the nearest-rank value: the k-th smallest,
// k the least integer >= p * n in exact arithmetic (k >= 1).  It is taken
// over the conducting voxels of the context (sigma > 0) carrying each label
// 0..L-1 (groups 0..L-1) and over every conducting voxel (group L).
//
// Method: an exact most-significant-digit radix select on the bit patterns
// of |E|.  For non-negative doubles the IEEE-754 bit pattern, read as an
// unsigned 64-bit integer, orders like the value, so selecting the k-th
// smallest key selects the k-th smallest value and the answer is one of the
// inputs, bit for bit.
//   1. count: voxels per group (one pass over the mask, E and the labels);
//   2. scatter: the keys of each group into a contiguous segment (a
//      conducting voxel lands in its label's segment and in the body's);
//   3. five rounds over the segments, one digit each (bits 62-50, 49-37,
//      36-24, 23-12, 11-0; bit 63 is the sign, 0 here): a shared-memory
//      histogram of the digit among the keys that still match the group's
//      chosen prefix, then one block per group walks its histogram to the
//      bucket holding the remaining rank and appends that digit.
// After the last round each group's prefix is the key of its answer.
#include <cstring>

#include "spfd_ctx.cuh"

namespace spfd {
namespace {

constexpr int PT = 256;              // threads per block
constexpr int PCT_TILE = PT * 8;     // voxels per block in count / scatter
constexpr int PCT_CHUNK = 4096;      // keys per block in the rounds
constexpr int PCT_BINS = 1 << 13;    // histogram bins (widest digit)
constexpr int PCT_ROUNDS = 5;
constexpr int PCT_SHIFT[PCT_ROUNDS] = {50, 37, 24, 12, 0};
constexpr int PCT_WIDTH[PCT_ROUNDS] = {13, 13, 13, 12, 12};
constexpr int PCT_MAX_LABELS = 2048;
constexpr int PCT_BAD_E = 1;         // status bit: negative or non-finite |E|
constexpr int PCT_BAD_RANK = 2;      // status bit: a rank fell outside its bucket

// Group of a voxel's label: the label itself when 0 <= label < L, else -1
// (the voxel then counts for the whole body only).
__device__ __forceinline__ int label_group(int lab, int L) {
  return (lab >= 0 && lab < L) ? lab : -1;
}

// Key of a conducting voxel's |E|: its bit pattern (+0 for -0), or flags it.
__device__ __forceinline__ unsigned long long e_key(double e, int *status) {
  if (!(e >= 0.0 && e <= 1.7976931348623157e308)) {
    atomicOr(status, PCT_BAD_E);
    return 0ull;
  }
  return e == 0.0 ? 0ull : (unsigned long long)__double_as_longlong(e);
}

// Adds v to cnt[g] once per group among the active lanes of the warp.
__device__ __forceinline__ unsigned warp_group_add(unsigned *cnt, int g, unsigned v,
                                                   unsigned active) {
  const unsigned peers = __match_any_sync(active, g);
  const int leader = __ffs(peers) - 1;
  const unsigned lane = threadIdx.x & 31;
  const unsigned rank = __popc(peers & ((1u << lane) - 1u));
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(&cnt[g], v * __popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + rank * v;
}

// Block b takes tiles b, b + grid, b + 2 grid, ... in both the count and the
// scatter pass (same grid), so each block's keys of a group form one run
// whose offset the scan fixes in advance.

// 1. Voxels per group and block: bcount[block][g] (groups 0..L-1 by label,
// L for the body).
__global__ void __launch_bounds__(PT)
k_pct_count(const unsigned char *__restrict__ mask, const double *__restrict__ E,
            const int *__restrict__ labels, long long nv, int L,
            unsigned *__restrict__ bcount, int *status) {
  extern __shared__ unsigned scnt[];  // L + 1
  for (int g = threadIdx.x; g <= L; g += PT) scnt[g] = 0;
  __syncthreads();
  const long long tiles = (nv + PCT_TILE - 1) / PCT_TILE;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * PCT_TILE;
    for (int q = 0; q < PCT_TILE / PT; ++q) {
      const long long v = base + q * PT + threadIdx.x;
      const bool cond = v < nv && mask[v];
      const unsigned active = __ballot_sync(0xffffffffu, cond);
      if (!cond) continue;
      e_key(__ldg(&E[v]), status);
      const int t = labels ? label_group(__ldg(&labels[v]), L) : -1;
      const unsigned inlab = __ballot_sync(active, t >= 0);
      if (t >= 0) warp_group_add(scnt, t, 1u, inlab);
      if ((threadIdx.x & 31) == __ffs(active) - 1) atomicAdd(&scnt[L], __popc(active));
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g <= L; g += PT) bcount[(size_t)blockIdx.x * (L + 1) + g] = scnt[g];
}

// 1b. One block per group: exclusive scan of the per-block counts over the
// blocks (boff), and the group's total (count).
__global__ void __launch_bounds__(PT)
k_pct_scan(const unsigned *__restrict__ bcount, int nblk, int G,
           unsigned long long *__restrict__ boff, unsigned long long *__restrict__ count) {
  __shared__ unsigned long long part[PT];
  const int g = blockIdx.x;
  const int per = (nblk + PT - 1) / PT;
  const int b0 = threadIdx.x * per, b1 = b0 + per < nblk ? b0 + per : nblk;
  unsigned long long s = 0;
  for (int b = b0; b < b1; ++b) s += bcount[(size_t)b * G + g];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < PT; o <<= 1) {
    const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned long long run = part[threadIdx.x] - s;
  for (int b = b0; b < b1; ++b) {
    boff[(size_t)b * G + g] = run;
    run += bcount[(size_t)b * G + g];
  }
  if (threadIdx.x == PT - 1) count[g] = part[PT - 1];
}

// 2. Keys into the segments: group g owns seg[off[g] .. off[g] + count[g]),
// in which block b's keys of group g start at boff[b][g].  No global atomics:
// a tile's keys take positions from shared-memory counters.
__global__ void __launch_bounds__(PT)
k_pct_scatter(const unsigned char *__restrict__ mask, const double *__restrict__ E,
              const int *__restrict__ labels, long long nv, int L,
              const long long *__restrict__ off, const unsigned long long *__restrict__ boff,
              const unsigned long long *__restrict__ count,
              unsigned long long *__restrict__ seg, int *status) {
  extern __shared__ unsigned char smem[];
  const int G = L + 1;
  unsigned *lc = (unsigned *)smem;   // this tile's counts
  unsigned *run = lc + G;            // this block's keys so far, per group
  constexpr int Q = PCT_TILE / PT;
  for (int g = threadIdx.x; g < G; g += PT) run[g] = 0;
  const long long tiles = (nv + PCT_TILE - 1) / PCT_TILE;
  const unsigned long long *bo = boff + (size_t)blockIdx.x * G;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * PCT_TILE;
    for (int g = threadIdx.x; g < G; g += PT) lc[g] = 0;
    __syncthreads();
    unsigned long long key[Q];
    int grp[Q];
    unsigned li[Q], lb[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const long long v = base + q * PT + threadIdx.x;
      const bool cond = v < nv && mask[v];
      const unsigned active = __ballot_sync(0xffffffffu, cond);
      grp[q] = -2;  // not conducting
      if (!cond) continue;
      key[q] = e_key(__ldg(&E[v]), status);
      const int t = labels ? label_group(__ldg(&labels[v]), L) : -1;
      grp[q] = t;
      const unsigned inlab = __ballot_sync(active, t >= 0);
      if (t >= 0) li[q] = warp_group_add(lc, t, 1u, inlab);
      lb[q] = warp_group_add(lc, L, 1u, active);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (grp[q] == -2) continue;
      // positions stay inside the segments when count and scatter saw the
      // same inputs; anything else is flagged instead of written
      if (grp[q] >= 0) {
        const int t = grp[q];
        const unsigned long long pos = bo[t] + run[t] + li[q];
        if (pos < count[t]) seg[off[t] + pos] = key[q];
        else atomicOr(status, PCT_BAD_RANK);
      }
      const unsigned long long pos = bo[L] + run[L] + lb[q];
      if (pos < count[L]) seg[off[L] + pos] = key[q];
      else atomicOr(status, PCT_BAD_RANK);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += PT) run[g] += lc[g];
    __syncthreads();
  }
}

// 3a. Digit histogram of the keys of one chunk that match their group's
// prefix above the digit; with cand_key set, the matching keys are also
// appended (with their group) to the candidate list.
__global__ void __launch_bounds__(PT)
k_pct_hist(const unsigned long long *__restrict__ seg, const int *__restrict__ chunk_group,
           const long long *__restrict__ chunk_begin, const long long *__restrict__ chunk_end,
           const unsigned long long *__restrict__ prefix, int shift, int width,
           unsigned *__restrict__ ghist, unsigned long long *__restrict__ cand_key,
           int *__restrict__ cand_grp, unsigned long long *__restrict__ cand_n) {
  __shared__ unsigned hist[PCT_BINS];
  const int g = chunk_group[blockIdx.x];
  const long long b = chunk_begin[blockIdx.x], e = chunk_end[blockIdx.x];
  const int hi = shift + width;
  const unsigned long long want = prefix[g] >> hi;
  const unsigned dmask = (1u << width) - 1u;
  for (int i = threadIdx.x; i < PCT_BINS; i += PT) hist[i] = 0;
  __syncthreads();
  for (long long i = b + threadIdx.x; i - threadIdx.x < e; i += PT) {
    const bool in = i < e;
    const unsigned long long k = in ? __ldg(&seg[i]) : 0ull;
    const bool match = in && (k >> hi) == want;
    const unsigned m = __ballot_sync(0xffffffffu, match);
    if (match) {
      warp_group_add(hist, (int)((k >> shift) & dmask), 1u, m);
      if (cand_key) {  // keep the matching keys for the later rounds
        const unsigned lane = threadIdx.x & 31;
        const int leader = __ffs(m) - 1;
        unsigned long long pos0 = 0;
        if ((int)lane == leader) pos0 = atomicAdd(cand_n, (unsigned long long)__popc(m));
        pos0 = __shfl_sync(m, pos0, leader);
        const unsigned long long pos = pos0 + __popc(m & ((1u << lane) - 1u));
        cand_key[pos] = k;
        cand_grp[pos] = g;
      }
    }
  }
  __syncthreads();
  unsigned *row = ghist + (size_t)g * PCT_BINS;
  for (int i = threadIdx.x; i <= (int)dmask; i += PT)
    if (hist[i]) atomicAdd(&row[i], hist[i]);
}

// 3c. The same over the compacted candidates (few keys): global-memory
// histogram counters, grid-stride over the *cand_n candidates.
__global__ void __launch_bounds__(PT)
k_pct_hist_cand(const unsigned long long *__restrict__ cand_key, const int *__restrict__ cand_grp,
                const unsigned long long *__restrict__ cand_n,
                const unsigned long long *__restrict__ prefix, int shift, int width,
                unsigned *__restrict__ ghist) {
  const unsigned long long n = *cand_n;
  const int hi = shift + width;
  const unsigned dmask = (1u << width) - 1u;
  for (unsigned long long i = (unsigned long long)blockIdx.x * PT + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * PT) {
    const unsigned long long k = cand_key[i];
    const int g = cand_grp[i];
    if ((k >> hi) == (prefix[g] >> hi))
      atomicAdd(&ghist[(size_t)g * PCT_BINS + ((k >> shift) & dmask)], 1u);
  }
}

// 3b. One block per group: the digit whose bucket holds the remaining rank;
// clears the group's histogram row for the next round.
__global__ void __launch_bounds__(PT)
k_pct_select(unsigned *__restrict__ ghist, const unsigned long long *__restrict__ count,
             unsigned long long *__restrict__ prefix, unsigned long long *__restrict__ rank,
             int shift, int width, int *status) {
  constexpr int PER = PCT_BINS / PT;  // 32 bins per thread
  __shared__ unsigned long long part[PT];
  __shared__ int found;
  const int g = blockIdx.x;
  if (count[g] == 0) return;
  unsigned *row = ghist + (size_t)g * PCT_BINS;
  const int nbin = 1 << width;
  unsigned h[PER];
  unsigned long long s = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bin = threadIdx.x * PER + q;
    h[q] = bin < nbin ? row[bin] : 0u;
    s += h[q];
  }
  part[threadIdx.x] = s;
  if (threadIdx.x == 0) found = 0;
  __syncthreads();
  // inclusive scan of the per-thread sums (Hillis-Steele over 256 entries)
  for (int o = 1; o < PT; o <<= 1) {
    const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  const unsigned long long r = rank[g];  // 1-based rank inside the current bucket
  const unsigned long long incl = part[threadIdx.x];
  const unsigned long long excl = incl - s;
  __syncthreads();
  if (excl < r && r <= incl) {
    unsigned long long cum = excl;
    for (int q = 0; q < PER; ++q) {
      if (cum + h[q] >= r) {
        const unsigned long long d = (unsigned long long)(threadIdx.x * PER + q);
        prefix[g] |= d << shift;
        rank[g] = r - cum;
        found = 1;
        break;
      }
      cum += h[q];
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int bin = threadIdx.x * PER + q;
    if (bin < nbin) row[bin] = 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !found) atomicOr(status, PCT_BAD_RANK);
}

// Least integer k >= p * n (exact; p in (0, 1] read as the binary fraction
// m / 2^s), at least 1; 0 when n = 0.
unsigned long long rank_of(double p, unsigned long long n) {
  if (n == 0) return 0;
  int e = 0;
  const double f = std::frexp(p, &e);
  const unsigned long long m = (unsigned long long)std::ldexp(f, 53);
  const int s = 53 - e;
  if (s >= 127) return 1;
  const unsigned __int128 x = (unsigned __int128)m * n;
  const unsigned __int128 one = 1;
  const unsigned long long k = (unsigned long long)((x + ((one << s) - 1)) >> s);
  return k < 1 ? 1 : k;
}

}  // namespace
}  // namespace spfd

using namespace spfd;

extern "C" spfd_status spfd_percentile(spfd_ctx *ctx, const double *E_dev,
                                       const int32_t *labels_dev, int n_labels, double p,
                                       double *values_host, int64_t *counts_host) {
  if (!ctx) return fail(SPFD_EINVAL, "ctx is NULL");
  if (!E_dev || !values_host || (n_labels > 0 && !labels_dev))
    return fail(SPFD_EINVAL, "null argument");
  if (n_labels < 0 || n_labels > PCT_MAX_LABELS)
    return fail(SPFD_EINVAL, "n_labels must be in 0..%d (got %d)", PCT_MAX_LABELS, n_labels);
  if (!(p > 0.0 && p <= 1.0)) return fail(SPFD_EINVAL, "p must be in (0, 1]");
  spfd_ctx *c = ctx;
  cudaStream_t st = c->stream;
  const int L = n_labels, G = L + 1;
  const long long nv = (long long)c->nx * c->ny * c->nz;
  // without labels every conducting voxel counts for the body only
  const int *lab = L > 0 ? (const int *)labels_dev : nullptr;
  // per-group scratch: counts, cursors, offsets, prefixes, ranks, status
  if (c->pct_gcap < G) {
    dfree(c, c->pct_small);
    dfree(c, c->pct_hist);
    TRY(dalloc(c, &c->pct_small, (size_t)5 * G + 1));
    TRY(dalloc(c, &c->pct_hist, (size_t)G * PCT_BINS));
    CU(cudaMemsetAsync(c->pct_hist, 0, (size_t)G * PCT_BINS * sizeof(unsigned), st));
    c->pct_gcap = G;
  }
  // cand_n (first entry of its slot): candidates kept after the first digit
  unsigned long long *cnt = c->pct_small, *cand_n = cnt + G, *pre = cand_n + G, *rk = pre + G;
  long long *off = (long long *)(rk + G);
  int *status = (int *)(off + G);
  CU(cudaMemsetAsync(c->pct_small, 0, ((size_t)5 * G + 1) * 8, st));
  const long long tiles = (nv + PCT_TILE - 1) / PCT_TILE;
  const int grid = (int)std::max(1LL, std::min(tiles, (long long)c->nsm * 8));
  if (c->pct_bcap < (long long)grid * G) {
    dfree(c, c->pct_bcnt);
    dfree(c, c->pct_boff);
    TRY(dalloc(c, &c->pct_bcnt, (size_t)grid * G));
    TRY(dalloc(c, &c->pct_boff, (size_t)grid * G));
    c->pct_bcap = (long long)grid * G;
  }
  const size_t sm_count = (size_t)G * sizeof(unsigned);
  // algorithmic bytes: the mask of every voxel, E and the label of each
  // conducting one (counted from the previous call; all voxels on the first)
  const double ncv = c->pct_nc > 0 ? (double)c->pct_nc : (double)nv;
  SPFD_LAUNCH(c, "percentile_count", false, 1, nv + 12.0 * ncv, 0,
              (k_pct_count<<<grid, PT, sm_count, st>>>(c->mask, E_dev, lab, nv, L, c->pct_bcnt,
                                                       status)));
  SPFD_LAUNCH(c, "percentile_count", false, 1, 12.0 * grid * G, 0,
              (k_pct_scan<<<G, PT, 0, st>>>(c->pct_bcnt, grid, G, c->pct_boff, cnt)));
  TRY(launch_check("percentile count"));
  std::vector<unsigned long long> hc(G);
  int hstatus = 0;
  CU(cudaMemcpyAsync(hc.data(), cnt, G * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st));
  TRY(sync_check(c, "percentile count"));
  if (hstatus & PCT_BAD_E)
    return fail(SPFD_EINVAL, "|E| holds a negative or non-finite value on a conducting voxel");
  // segments, ranks and the chunk table of the rounds
  std::vector<long long> hoff(G), hrk(G);
  std::vector<int> cg;
  std::vector<long long> cb, ce;
  long long total = 0;
  for (int g = 0; g < G; ++g) {
    hoff[g] = total;
    hrk[g] = (long long)rank_of(p, hc[g]);
    for (long long b = total; b < total + (long long)hc[g]; b += PCT_CHUNK) {
      cg.push_back(g);
      cb.push_back(b);
      ce.push_back(std::min(b + PCT_CHUNK, total + (long long)hc[g]));
    }
    total += (long long)hc[g];
  }
  const int nch = (int)cg.size();
  if (c->pct_keycap < total) {
    dfree(c, c->pct_keys);
    dfree(c, c->pct_cand);
    dfree(c, c->pct_candg);
    TRY(dalloc(c, &c->pct_keys, (size_t)total));
    TRY(dalloc(c, &c->pct_cand, (size_t)total));
    TRY(dalloc(c, &c->pct_candg, (size_t)total));
    c->pct_keycap = total;
  }
  if (c->pct_chcap < nch) {
    dfree(c, c->pct_chunks);
    TRY(dalloc(c, &c->pct_chunks, (size_t)3 * nch));
    c->pct_chcap = nch;
  }
  // host staging (pinned, kept by the context): offsets, ranks, chunk table
  const size_t stage_n = (size_t)2 * G + 3 * (size_t)nch;
  if (c->pct_hstage_n < stage_n) {
    TRY(halloc(c, &c->pct_hstage, stage_n));
    c->pct_hstage_n = stage_n;
  }
  long long *hs = c->pct_hstage;
  memcpy(hs, hoff.data(), G * 8);
  memcpy(hs + G, hrk.data(), G * 8);
  long long *hch = hs + 2 * G;
  int *hcg = (int *)(hch + 2 * nch);
  for (int q = 0; q < nch; ++q) {
    hch[q] = cb[q];
    hch[nch + q] = ce[q];
    hcg[q] = cg[q];
  }
  CU(cudaMemcpyAsync(off, hs, G * 8, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(rk, hs + G, G * 8, cudaMemcpyHostToDevice, st));
  long long *dcb = c->pct_chunks, *dce = dcb + nch;
  int *dcg = (int *)(dce + nch);
  if (nch > 0) {
    CU(cudaMemcpyAsync(dcb, hch, (size_t)2 * nch * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dcg, hcg, (size_t)nch * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  const size_t sm_scatter = (size_t)2 * G * sizeof(unsigned);
  c->pct_nc = (long long)hc[L];
  SPFD_LAUNCH(c, "percentile_scatter", false, 1, nv + 12.0 * hc[L] + 8.0 * total, 0,
              (k_pct_scatter<<<grid, PT, sm_scatter, st>>>(c->mask, E_dev, lab, nv, L, off,
                                                           c->pct_boff, cnt, c->pct_keys,
                                                           status)));
  TRY(launch_check("percentile scatter"));
  // rounds 0 and 1 read every key (round 1 keeps those that match the first
  // digit); rounds 2-4 read only those candidates
  for (int r = 0; r < PCT_ROUNDS && nch > 0; ++r) {
    if (r < 2) {
      SPFD_LAUNCH(c, "percentile_hist", false, 1, 8.0 * total, 0,
                  (k_pct_hist<<<nch, PT, 0, st>>>(
                      c->pct_keys, dcg, dcb, dce, pre, PCT_SHIFT[r], PCT_WIDTH[r], c->pct_hist,
                      r == 1 ? c->pct_cand : nullptr, c->pct_candg, cand_n)));
    } else {
      SPFD_LAUNCH(c, "percentile_hist", false, 1, 0, 0,
                  (k_pct_hist_cand<<<c->nsm * 4, PT, 0, st>>>(c->pct_cand, c->pct_candg, cand_n,
                                                              pre, PCT_SHIFT[r], PCT_WIDTH[r],
                                                              c->pct_hist)));
    }
    SPFD_LAUNCH(c, "percentile_select", false, 1, 8.0 * G * (1 << PCT_WIDTH[r]), 0,
                (k_pct_select<<<G, PT, 0, st>>>(c->pct_hist, cnt, pre, rk, PCT_SHIFT[r],
                                                PCT_WIDTH[r], status)));
  }
  TRY(launch_check("percentile rounds"));
  std::vector<unsigned long long> hpre(G);
  CU(cudaMemcpyAsync(hpre.data(), pre, G * 8, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, st));
  TRY(sync_check(c, "percentile"));
  TRY(prof_flush(c));
  if (hstatus & PCT_BAD_RANK)
    return fail(SPFD_EINTERNAL, "percentile selection lost its rank (|E| or labels "
                                "changed during the call?)");
  for (int g = 0; g < G; ++g) {
    double v = NAN;
    if (hc[g]) memcpy(&v, &hpre[g], 8);
    values_host[g] = v;
    if (counts_host) counts_host[g] = (int64_t)hc[g];
  }
  return SPFD_OK;
}
