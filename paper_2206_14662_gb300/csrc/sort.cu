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
// Warp-mates with equal keys are combined with __match_any_sync so that one
// atomic serves a whole group.
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ int cell_key(int cell, int nz) {
  return cell < 0 ? -1 : (cell >> 16) * nz + (cell & 0xFFFF);
}

template <typename Real>
__global__ void k_sort_hist(const int* __restrict__ cell, const DevState* st,
                            int* count, int nz) {
  const long long n = st->n_slots;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
       base += (long long)gridDim.x * blockDim.x) {
    const long long p = base + threadIdx.x;
    const int key = p < n ? cell_key(cell[p], nz) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    if (key >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(count + key, __popc(peers));
  }
}

// exclusive scan of count[0..n) in place, one block of 1024 threads; the
// total goes to st->n_live
__global__ void __launch_bounds__(1024) k_sort_scan(int* count, int n, DevState* st) {
  __shared__ int part[1024];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    const int c = count[i];
    count[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) st->n_live = part[blockDim.x - 1];
}

template <typename Real>
__global__ void k_sort_scatter(Soa<Real> src, Soa<Real> dst, const DevState* st,
                               int* cursor, int nz) {
  const long long n = st->n_slots;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
       base += (long long)gridDim.x * blockDim.x) {
    const long long p = base + threadIdx.x;
    const int c = p < n ? src.cell[p] : -1;
    const int key = cell_key(c, nz);
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int slot = 0;
    if (key >= 0 && lane == leader) slot = atomicAdd(cursor + key, __popc(peers));
    slot = __shfl_sync(0xffffffffu, slot, leader);
    if (key >= 0) {
      const int q = slot + __popc(peers & ((1u << lane) - 1u));
      dst.cell[q] = c;
      dst.offr[q] = src.offr[p];
      dst.offz[q] = src.offz[p];
      dst.vr[q] = src.vr[p];
      dst.vt[q] = src.vt[p];
      dst.vz[q] = src.vz[p];
      dst.uid[q] = src.uid[p];
    }
  }
}

__global__ void k_sort_commit(DevState* st) { st->n_slots = st->n_live; }

template <typename Real>
void launch_sort(const Soa<Real>& src, const Soa<Real>& dst, DevState* st,
                 int* cell_count, int ncells, int nz, int grid,
                 cudaStream_t stream) {
  cudaMemsetAsync(cell_count, 0, (size_t)ncells * sizeof(int), stream);
  k_sort_hist<Real><<<grid, 256, 0, stream>>>(src.cell, st, cell_count, nz);
  k_sort_scan<<<1, 1024, 0, stream>>>(cell_count, ncells, st);
  k_sort_scatter<Real><<<grid, 256, 0, stream>>>(src, dst, st, cell_count, nz);
  k_sort_commit<<<1, 1, 0, stream>>>(st);
}

template void launch_sort<float>(const Soa<float>&, const Soa<float>&, DevState*, int*, int,
                                 int, int, cudaStream_t);
template void launch_sort<double>(const Soa<double>&, const Soa<double>&, DevState*, int*, int,
                                  int, int, cudaStream_t);

}  // namespace pic
