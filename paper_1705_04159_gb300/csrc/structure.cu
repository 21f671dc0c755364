// structure.cu -- rating structure on the device (built once per sampler).
//
// Algorithm 1 loops over "all movies" and "all users" and, for each, over
// the ratings of that row or column.  This file builds both views of R:
// row-compressed (users) and column-compressed (movies), each with a stable
// order (a row's ratings keep their input order), ratings centred by their
// mean, and each side's rows ordered by degree (largest first, ties by row
// id) for the degree-binned launch.  All orders are produced by a stable LSD
// radix sort written here, so the structure is bit-for-bit reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bpmf_impl.cuh"

namespace gb {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;
constexpr int kSortWarps = kSortThreads / 32;

// Per-tile digit histogram, stored digit-major: counts[d * tiles + tile].
__global__ void radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                           int32_t* __restrict__ counts, int tiles) {
  __shared__ int32_t hist[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t e = base + (int64_t)j * kSortThreads + threadIdx.x;
    if (e < n) atomicAdd(&hist[(keys[e] >> shift) & (kRadix - 1)], 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
    counts[(int64_t)i * tiles + blockIdx.x] = hist[i];
}

// Stable scatter of one tile: items are visited in input order (round j,
// then thread id); an item's slot is the tile's base offset for its digit
// plus the number of earlier items of the tile with the same digit.
__global__ void radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                              uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                              int shift, const int32_t* __restrict__ offs, int tiles) {
  __shared__ int32_t running[kRadix];
  __shared__ int32_t warp_cnt[kSortWarps][kRadix + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x)
    running[i] = offs[(int64_t)i * tiles + blockIdx.x];
  for (int i = threadIdx.x; i < kSortWarps * (kRadix + 1); i += blockDim.x)
    (&warp_cnt[0][0])[i] = 0;
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t e = base + (int64_t)j * kSortThreads + threadIdx.x;
    const bool ok = e < n;
    const uint32_t k = ok ? kin[e] : 0u;
    const int32_t v = ok ? vin[e] : 0;
    const int d = ok ? (int)((k >> shift) & (kRadix - 1)) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & below);
    if (lane == __ffs(peers) - 1) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      int pos = running[d] + rank;
      for (int w = 0; w < warp; ++w) pos += warp_cnt[w][d];
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kRadix + 1; i += blockDim.x) {
      int s = 0;
      for (int w = 0; w < kSortWarps; ++w) {
        s += warp_cnt[w][i];
        warp_cnt[w][i] = 0;
      }
      if (i < kRadix) running[i] += s;
    }
    __syncthreads();
  }
}

// Exclusive scan of int32 in blocks of 2048 (256 threads x 8 items); the
// block totals go to `sums` for the next level.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tiles(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                           int32_t* __restrict__ sums) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t tot = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    tot += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  int32_t wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
  int32_t run = wbase + inc - tot;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = wbase + inc;
}

__global__ void scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const int32_t o = offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t e = i + (int64_t)k * kScanThreads;
    if (e < n) out[e] += o;
  }
}

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return BPMF_OK;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int32_t* sums = nullptr;
  int32_t* sums_scanned = nullptr;
  BPMF_CUDA_CHECK(cudaMallocAsync(&sums, sizeof(int32_t) * tiles, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&sums_scanned, sizeof(int32_t) * tiles, st));
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums);
  BPMF_CUDA_CHECK(cudaGetLastError());
  if (tiles > 1) {
    int rc = exclusive_scan_i32(sums, sums_scanned, tiles, st);
    if (rc != BPMF_OK) return rc;
    scan_add<<<(unsigned)tiles, kScanThreads, 0, st>>>(out, n, sums_scanned);
    BPMF_CUDA_CHECK(cudaGetLastError());
  }
  BPMF_CUDA_CHECK(cudaFreeAsync(sums, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(sums_scanned, st));
  return BPMF_OK;
}

__global__ void iota_i32(int32_t* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

__global__ void check_indices(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                              int64_t n, int64_t M, int64_t N, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = row[e], c = col[e];
    if (r < 0 || r >= M || c < 0 || c >= N) atomicOr(status, kStatusIndex);
  }
}

__global__ void check_finite(const float* __restrict__ v, int64_t n, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[e])) atomicOr(status, kStatusValue);
}

// Fixed-shape FP64 sum: block b sums elements b, b + G*256, ... in a fixed
// pattern, then one thread adds the block sums in block order.
constexpr int kMeanBlocks = 512;
__global__ void sum_partials(const float* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double ws[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}
__global__ void sum_final(const double* __restrict__ part, int nparts, int64_t n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += part[i];
    out[0] = n > 0 ? t / (double)n : 0.0;
  }
}

// key of entry e for the sort of one side
__global__ void gather_keys(const int32_t* __restrict__ key, uint32_t* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (uint32_t)key[e];
}

// idx[p] = other[src[p]], val[p] = val_in[src[p]] - mean (rounded once)
__global__ void gather_entries(const int32_t* __restrict__ src, const int32_t* __restrict__ other,
                               const float* __restrict__ vin, double mean, int32_t* __restrict__ idx,
                               float* __restrict__ val, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = src[p];
    idx[p] = other[e];
    val[p] = (float)((double)vin[e] - mean);
  }
}

// ptr[r] = first position of key r in the sorted keys (lower bound)
__global__ void row_pointers(const uint32_t* __restrict__ sorted, int64_t n, int64_t R,
                             int64_t* __restrict__ ptr) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= R;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)sorted[mid] < r) lo = mid + 1;
      else hi = mid;
    }
    ptr[r] = lo;
  }
}

__global__ void degree_keys(const int64_t* __restrict__ ptr, int64_t R, uint32_t maxdeg,
                            uint32_t* __restrict__ keys) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x)
    keys[r] = maxdeg - (uint32_t)(ptr[r + 1] - ptr[r]);
}

__global__ void max_degree(const int64_t* __restrict__ ptr, int64_t R, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)(ptr[r + 1] - ptr[r]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535LL * 16) g = 65535LL * 16;
  return (unsigned)g;
}

}  // namespace

// Stable sort of (key, value) pairs by key, LSD with 8-bit digits; passes
// stop once every key bit up to max_key has been consumed.
int sort_pairs_u32(uint32_t* keys_io, int32_t* vals_io, uint32_t* keys_out, int32_t* vals_out,
                   int64_t n, uint32_t max_key, cudaStream_t st) {
  if (n <= 0) return BPMF_OK;
  int bits = 0;
  while (bits < 32 && (max_key >> bits) != 0u) ++bits;
  const int passes = bits == 0 ? 1 : (bits + 7) / 8;
  const int tiles = (int)((n + kSortTile - 1) / kSortTile);
  uint32_t *ka = keys_io, *kb = keys_out;
  int32_t *va = vals_io, *vb = vals_out, *counts = nullptr, *offs = nullptr;
  BPMF_CUDA_CHECK(cudaMallocAsync(&counts, sizeof(int32_t) * (int64_t)kRadix * tiles, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&offs, sizeof(int32_t) * (int64_t)kRadix * tiles, st));
  for (int p = 0; p < passes; ++p) {
    radix_hist<<<tiles, kSortThreads, 0, st>>>(ka, n, 8 * p, counts, tiles);
    BPMF_CUDA_CHECK(cudaGetLastError());
    int rc = exclusive_scan_i32(counts, offs, (int64_t)kRadix * tiles, st);
    if (rc != BPMF_OK) return rc;
    radix_scatter<<<tiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, 8 * p, offs, tiles);
    BPMF_CUDA_CHECK(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // after an even number of passes the result is back in the input pair
  if (ka != keys_out) {
    BPMF_CUDA_CHECK(cudaMemcpyAsync(keys_out, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    BPMF_CUDA_CHECK(cudaMemcpyAsync(vals_out, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  }
  BPMF_CUDA_CHECK(cudaFreeAsync(counts, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(offs, st));
  return BPMF_OK;
}

double device_mean(const float* d_val, int64_t n, double* d_red, cudaStream_t st, int* err) {
  *err = BPMF_OK;
  if (n <= 0) return 0.0;
  sum_partials<<<kMeanBlocks, 256, 0, st>>>(d_val, n, d_red);
  sum_final<<<1, 32, 0, st>>>(d_red, kMeanBlocks, n, d_red + kMeanBlocks);
  double m = 0.0;
  if (cudaMemcpyAsync(&m, d_red + kMeanBlocks, sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("device_mean: %s", cudaGetErrorString(cudaGetLastError()));
    *err = BPMF_ECUDA;
  }
  return m;
}

int order_rows_by_degree(Handle* h, int s) {
  SideDev& sd = h->side[s];
  cudaStream_t st = h->stream;
  const int64_t R = sd.R;
  unsigned long long* dmax = nullptr;
  BPMF_CUDA_CHECK(cudaMallocAsync(&dmax, sizeof(unsigned long long), st));
  BPMF_CUDA_CHECK(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st));
  max_degree<<<grid_for(R, 256), 256, 0, st>>>(sd.ptr, R, dmax);
  BPMF_CUDA_CHECK(cudaGetLastError());
  unsigned long long maxdeg = 0;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(&maxdeg, dmax, sizeof(maxdeg), cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  BPMF_CUDA_CHECK(cudaFreeAsync(dmax, st));
  sd.max_deg = (int64_t)maxdeg;
  uint32_t* keys = nullptr;
  uint32_t* keys_sorted = nullptr;
  int32_t* ids = nullptr;
  BPMF_CUDA_CHECK(cudaMallocAsync(&keys, sizeof(uint32_t) * R, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&keys_sorted, sizeof(uint32_t) * R, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&ids, sizeof(int32_t) * R, st));
  degree_keys<<<grid_for(R, 256), 256, 0, st>>>(sd.ptr, R, (uint32_t)maxdeg, keys);
  iota_i32<<<grid_for(R, 256), 256, 0, st>>>(ids, R);
  BPMF_CUDA_CHECK(cudaGetLastError());
  BPMF_TRY(sort_pairs_u32(keys, ids, keys_sorted, sd.perm, R, (uint32_t)maxdeg, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(keys, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(keys_sorted, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(ids, st));
  return BPMF_OK;
}

int build_structure(Handle* h, const int32_t* d_row, const int32_t* d_col, const float* d_val) {
  cudaStream_t st = h->stream;
  const int64_t nnz = h->nnz;
  if (nnz > 0) {
    check_indices<<<grid_for(nnz, 256), 256, 0, st>>>(d_row, d_col, nnz, h->M, h->N, h->status);
    check_finite<<<grid_for(nnz, 256), 256, 0, st>>>(d_val, nnz, h->status);
    BPMF_CUDA_CHECK(cudaGetLastError());
    int st_h = 0;
    BPMF_CUDA_CHECK(cudaMemcpyAsync(&st_h, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
    if (st_h & (kStatusIndex | kStatusValue)) {
      BPMF_CUDA_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
      set_error(st_h & kStatusIndex ? "bpmf_init: a rating index is outside [0, M) x [0, N)"
                                    : "bpmf_init: a rating is not finite");
      return BPMF_EINVAL;
    }
  }
  int err = BPMF_OK;
  h->mean = device_mean(d_val, nnz, h->red, st, &err);
  if (err != BPMF_OK) return err;

  uint32_t* keys = nullptr;
  uint32_t* keys_sorted = nullptr;
  int32_t* ids = nullptr;
  int32_t* src = nullptr;
  const int64_t n_alloc = nnz > 0 ? nnz : 1;
  BPMF_CUDA_CHECK(cudaMallocAsync(&keys, sizeof(uint32_t) * n_alloc, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&keys_sorted, sizeof(uint32_t) * n_alloc, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&ids, sizeof(int32_t) * n_alloc, st));
  BPMF_CUDA_CHECK(cudaMallocAsync(&src, sizeof(int32_t) * n_alloc, st));
  for (int s = 0; s < 2; ++s) {
    SideDev& sd = h->side[s];
    const int32_t* key = s == BPMF_USERS ? d_row : d_col;
    const int32_t* other = s == BPMF_USERS ? d_col : d_row;
    if (nnz > 0) {
      gather_keys<<<grid_for(nnz, 256), 256, 0, st>>>(key, keys, nnz);
      iota_i32<<<grid_for(nnz, 256), 256, 0, st>>>(ids, nnz);
      BPMF_CUDA_CHECK(cudaGetLastError());
      BPMF_TRY(sort_pairs_u32(keys, ids, keys_sorted, src, nnz, (uint32_t)(sd.R - 1), st));
      gather_entries<<<grid_for(nnz, 256), 256, 0, st>>>(src, other, d_val, h->mean, sd.idx,
                                                          sd.val, nnz);
      BPMF_CUDA_CHECK(cudaGetLastError());
    }
    row_pointers<<<grid_for(sd.R + 1, 256), 256, 0, st>>>(keys_sorted, nnz, sd.R, sd.ptr);
    BPMF_CUDA_CHECK(cudaGetLastError());
    BPMF_TRY(order_rows_by_degree(h, s));
  }
  BPMF_CUDA_CHECK(cudaFreeAsync(keys, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(keys_sorted, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(ids, st));
  BPMF_CUDA_CHECK(cudaFreeAsync(src, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  return BPMF_OK;
}

}  // namespace gb

namespace gb {
namespace {

__global__ void gather_test(const int32_t* __restrict__ src, const int32_t* __restrict__ row,
                            const int32_t* __restrict__ col, const float* __restrict__ val,
                            int32_t* __restrict__ trow, int32_t* __restrict__ tcol,
                            float* __restrict__ tval, int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = src[p];
    trow[p] = row[e];
    tcol[p] = col[e];
    tval[p] = val[e];
  }
}

}  // namespace

int validate_pairs(Handle* h, const int32_t* d_row, const int32_t* d_col, int64_t n) {
  if (n <= 0) return BPMF_OK;
  check_indices<<<grid_for(n, 256), 256, 0, h->stream>>>(d_row, d_col, n, h->M, h->N, h->status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

int sort_test_set(Handle* h, const int32_t* d_row, const int32_t* d_col, const float* d_val,
                  int64_t n, uint32_t* keys, uint32_t* keys_sorted, int32_t* ids, int32_t* src) {
  cudaStream_t st = h->stream;
  BPMF_TRY(validate_pairs(h, d_row, d_col, n));
  check_finite<<<grid_for(n, 256), 256, 0, st>>>(d_val, n, h->status);
  BPMF_CUDA_CHECK(cudaGetLastError());
  int st_h = 0;
  BPMF_CUDA_CHECK(cudaMemcpyAsync(&st_h, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  BPMF_CUDA_CHECK(cudaStreamSynchronize(st));
  if (st_h & (kStatusIndex | kStatusValue)) {
    BPMF_CUDA_CHECK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    set_error(st_h & kStatusIndex ? "bpmf_set_test: a test index is outside [0, M) x [0, N)"
                                  : "bpmf_set_test: a test rating is not finite");
    return BPMF_EINVAL;
  }
  gather_keys<<<grid_for(n, 256), 256, 0, st>>>(d_row, keys, n);
  iota_i32<<<grid_for(n, 256), 256, 0, st>>>(ids, n);
  BPMF_CUDA_CHECK(cudaGetLastError());
  BPMF_TRY(sort_pairs_u32(keys, ids, keys_sorted, src, n, (uint32_t)(h->M - 1), st));
  gather_test<<<grid_for(n, 256), 256, 0, st>>>(src, d_row, d_col, d_val, h->trow, h->tcol,
                                                 h->tval, n);
  BPMF_CUDA_CHECK(cudaGetLastError());
  return BPMF_OK;
}

}  // namespace gb
