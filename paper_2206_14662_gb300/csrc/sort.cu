// sort.cu -- periodic counting sort of the particle store by cell.
//
// Sorting keeps the particles of one block within a few cells of each
// other, so the fused kernel's gathers hit L1 and its deposits fit one
// shared-memory tile.  The same pass drops absorbed particles (holes) and
// merges the children appended since the last sort.
//   1. histogram of live particles per cell (key ir * nz + iz)
//   2. exclusive scan of the histogram (one block); the total becomes the
//      new slot count
//   3. scatter of every live particle to its cell's next free slot in the
//      other buffer set (slot order within a cell is not specified)
// The store is nearly sorted already (it was sorted sort_every steps ago),
// so runs of equal keys in consecutive lanes are common: one shuffle and
// one ballot find each run, and the run's first lane does one atomic for
// the whole run.
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ int cell_key(int cell, int nz) {
  return cell < 0 ? -1 : (cell >> 16) * nz + (cell & 0xFFFF);
}

// Runs of equal keys among the lanes of a warp: whether this lane starts a
// run, the lane starting its run, and (for run starts) the run's length.
struct Run {
  bool head;
  int first;
  int len;
};
__device__ __forceinline__ Run lane_run(int key, int lane) {
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const unsigned le = 0xffffffffu >> (31 - lane);   // lanes 0..lane
  Run r;
  r.head = head;
  r.first = 31 - __clz(heads & le);
  const unsigned above = heads & ~le;
  r.len = (above ? __ffs(above) - 1 : 32) - lane;
  return r;
}

// histogram: each thread takes four consecutive slots (one 16-byte load;
// the store is allocated in whole chunks of 1024 slots, so the vector never
// leaves it), runs are found among the lanes for each of the four
constexpr int kSortThreads = 256;
constexpr int kSortChunk = 4 * kSortThreads;

__device__ __forceinline__ void hist_group(const int* __restrict__ cell, int n, int p0,
                                           int* count, int nz, int lane) {
  const int4 c = *reinterpret_cast<const int4*>(cell + p0);
  const int cs[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int key = p0 + k < n ? cell_key(cs[k], nz) : -1;
    const Run r = lane_run(key, lane);
    if (key >= 0 && r.head) atomicAdd(count + key, r.len);
  }
}

template <typename Real>
__global__ void __launch_bounds__(kSortThreads)
k_sort_hist(const int* __restrict__ cell, const DevState* st, int* count, int nz) {
  const int n = (int)st->n_slots;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * kSortChunk; base < n; base += gridDim.x * kSortChunk)
    hist_group(cell, n, base + 4 * threadIdx.x, count, nz, lane);
}

// a batch: the chunks of all segments in one launch; simulation k counts
// into count + k * count_stride
__global__ void __launch_bounds__(kSortThreads)
k_sort_hist_batch(const int* __restrict__ cell, const DevState* st, const SegInfo* seg, int nsim,
                  int* count, int count_stride, int nz) {
  __shared__ int first[kMaxSims + 1];
  __shared__ long long nslots[kMaxSims];
  chunk_table(st, nsim, kSortChunk, first, nslots);
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < first[nsim]; c += gridDim.x) {
    const int sim = chunk_owner(first, nsim, c);
    const int p0 = (c - first[sim]) * kSortChunk + 4 * threadIdx.x;
    hist_group(cell + seg[sim].base, (int)nslots[sim], p0, count + (size_t)sim * count_stride,
               nz, lane);
  }
}

// exclusive scan of count[0..n) in place, one block of 1024 threads, each
// owning a contiguous stretch of whole int4 vectors (count is allocated in
// whole multiples of 4096 entries, the tail beyond n zero); the total goes
// to st->n_live.  Block k scans simulation k's counts (count + k *
// count_stride, st + k).
__global__ void __launch_bounds__(1024) k_sort_scan(int* count, int n, DevState* st,
                                                    int count_stride) {
  count += (size_t)blockIdx.x * count_stride;
  st += blockIdx.x;
  __shared__ int part[1024];
  const int n4 = (n + 4095) / 4096 * 1024;     // int4 vectors, whole per thread
  const int per = n4 / 1024;                   // vectors per thread
  int4* c4 = reinterpret_cast<int4*>(count) + (size_t)threadIdx.x * per;
  int s = 0;
  for (int i = 0; i < per; ++i) {
    const int4 v = c4[i];
    s += v.x + v.y + v.z + v.w;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
  for (int i = 0; i < per; ++i) {
    const int4 v = c4[i];
    int4 o;
    o.x = run; run += v.x;
    o.y = run; run += v.y;
    o.z = run; run += v.z;
    o.w = run; run += v.w;
    c4[i] = o;
  }
  if (threadIdx.x == 1023) st->n_live = part[1023];
}

// scatter: a block takes 1024 consecutive slots in four passes of 256
// lane-consecutive slots (coalesced loads; runs of equal cells fall on
// consecutive lanes, which then write consecutive destination slots); each
// live particle goes to its cell's next free slot in the other buffer set.
// A thread first loads its four particles, then claims the four runs'
// slots (independent atomics in flight together), then stores, so the
// loads and the atomics' round trips overlap instead of alternating.
template <typename Real>
__device__ __forceinline__ void scatter_group(const Soa<Real>& src, const Soa<Real>& dst, int n,
                                              int base, int* cursor, int nz, int lane) {
  int c[4], key[4];
  Real fr[4], fz[4], vr[4], vt[4], vz[4];
  unsigned id[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int p = base + k * kSortThreads + (int)threadIdx.x;
    c[k] = p < n ? src.cell[p] : -1;
    key[k] = cell_key(c[k], nz);
    if (key[k] >= 0) {
      fr[k] = src.offr[p];
      fz[k] = src.offz[p];
      vr[k] = src.vr[p];
      vt[k] = src.vt[p];
      vz[k] = src.vz[p];
      id[k] = src.uid[p];
    }
  }
  Run r[4];
  int slot[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r[k] = lane_run(key[k], lane);
    slot[k] = 0;
    if (key[k] >= 0 && r[k].head) slot[k] = atomicAdd(cursor + key[k], r[k].len);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int s0 = __shfl_sync(0xffffffffu, slot[k], r[k].first);
    if (key[k] >= 0) {
      const int q = s0 + (lane - r[k].first);
      dst.cell[q] = c[k];
      dst.offr[q] = fr[k];
      dst.offz[q] = fz[k];
      dst.vr[q] = vr[k];
      dst.vt[q] = vt[k];
      dst.vz[q] = vz[k];
      dst.uid[q] = id[k];
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(kSortThreads)
k_sort_scatter(Soa<Real> src, Soa<Real> dst, const DevState* st, int* cursor, int nz) {
  const int n = (int)st->n_slots;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * kSortChunk; base < n; base += gridDim.x * kSortChunk)
    scatter_group(src, dst, n, base, cursor, nz, lane);
}

// a batch: simulation k's particles stay in its segment (the same base in
// both buffer sets)
template <typename Real>
__global__ void __launch_bounds__(kSortThreads)
k_sort_scatter_batch(Soa<Real> src, Soa<Real> dst, const DevState* st, const SegInfo* seg,
                     int nsim, int* cursor, int count_stride, int nz) {
  __shared__ int first[kMaxSims + 1];
  __shared__ long long nslots[kMaxSims];
  chunk_table(st, nsim, kSortChunk, first, nslots);
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < first[nsim]; c += gridDim.x) {
    const int sim = chunk_owner(first, nsim, c);
    const long long b = seg[sim].base;
    scatter_group(soa_offset(src, b), soa_offset(dst, b), (int)nslots[sim],
                  (c - first[sim]) * kSortChunk, cursor + (size_t)sim * count_stride, nz, lane);
  }
}

__global__ void k_sort_commit(DevState* st, int nsim) {
  for (int k = threadIdx.x; k < nsim; k += blockDim.x) st[k].n_slots = st[k].n_live;
}

template <typename Real>
void launch_sort(const Soa<Real>& src, const Soa<Real>& dst, DevState* st,
                 int* cell_count, int ncells, int nz, int grid,
                 cudaStream_t stream) {
  cudaMemsetAsync(cell_count, 0, (size_t)(ncells + 4095) / 4096 * 4096 * sizeof(int), stream);
  k_sort_hist<Real><<<grid, kSortThreads, 0, stream>>>(src.cell, st, cell_count, nz);
  k_sort_scan<<<1, 1024, 0, stream>>>(cell_count, ncells, st, 0);
  k_sort_scatter<Real><<<grid, kSortThreads, 0, stream>>>(src, dst, st, cell_count, nz);
  k_sort_commit<<<1, 1, 0, stream>>>(st, 1);
}

template <typename Real>
void launch_sort_batch(const Soa<Real>& src, const Soa<Real>& dst, DevState* st,
                       const SegInfo* seg, int nsim, int* cell_count, int ncells, int nz,
                       int grid, cudaStream_t stream) {
  const int stride = (ncells + 4095) / 4096 * 4096;
  cudaMemsetAsync(cell_count, 0, (size_t)nsim * stride * sizeof(int), stream);
  k_sort_hist_batch<<<grid, kSortThreads, 0, stream>>>(src.cell, st, seg, nsim, cell_count,
                                                       stride, nz);
  k_sort_scan<<<nsim, 1024, 0, stream>>>(cell_count, ncells, st, stride);
  k_sort_scatter_batch<Real><<<grid, kSortThreads, 0, stream>>>(src, dst, st, seg, nsim,
                                                                cell_count, stride, nz);
  k_sort_commit<<<1, 256, 0, stream>>>(st, nsim);
}

template void launch_sort<float>(const Soa<float>&, const Soa<float>&, DevState*, int*, int,
                                 int, int, cudaStream_t);
template void launch_sort<double>(const Soa<double>&, const Soa<double>&, DevState*, int*, int,
                                  int, int, cudaStream_t);
template void launch_sort_batch<float>(const Soa<float>&, const Soa<float>&, DevState*,
                                       const SegInfo*, int, int*, int, int, int, cudaStream_t);
template void launch_sort_batch<double>(const Soa<double>&, const Soa<double>&, DevState*,
                                        const SegInfo*, int, int*, int, int, int, cudaStream_t);

}  // namespace pic
