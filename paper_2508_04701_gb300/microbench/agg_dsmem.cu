// Microbenchmark of where the probe pass's aggregate updates can go: throughput of 64-bit
// atomics on random 32-byte slots {sum, count, min, max} of an aggregate table, 180M updates
// (the joined rows of the 600M-row query), one update = add, add, min, max (kOps = 4) or
// add, add (kOps = 2):
//   L2    : global reductions into a 262144-slot table in L2 (what the fused probe does)
//   remote: shared-memory atomics on other CTAs of a thread-block cluster (the table split
//           over the cluster's ranks, reached through distributed shared memory)
//   local : shared-memory atomics on the CTA's own slice (no remote traffic)
// Also prints how many clusters of 8 and 16 CTAs fit with ~100 and ~200 KB of shared memory.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o agg_dsmem agg_dsmem.cu && ./agg_dsmem
#include <cooperative_groups.h>
#include <cstdio>
#include <cstdlib>
#include <cstdint>

namespace cg = cooperative_groups;

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); exit(1); } } while (0)

__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct __align__(32) Agg { unsigned long long sum, cnt; long long mn, mx; };

template <int kOps>
__device__ __forceinline__ void upd(Agg* a, int64_t v) {
  atomicAdd(&a->sum, (unsigned long long)v);
  atomicAdd(&a->cnt, 1ull);
  if (kOps == 4) {
    atomicMin(&a->mn, (long long)v);
    atomicMax(&a->mx, (long long)v);
  }
}

template <int kOps>
__global__ void l2_kernel(Agg* tab, uint32_t slots, int64_t updates_per_thread) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (int64_t k = 0; k < updates_per_thread; ++k) {
    const uint64_t h = mix(tid * 1000003ull + k);
    const uint32_t s = (uint32_t)(((h >> 32) * (uint64_t)slots) >> 32);  // < slots
    upd<kOps>(&tab[s], (int64_t)(h & 0xFFFFFF));
  }
}

// slots_per_cta slots in each CTA's dynamic shared memory; a random slot of the cluster's
// table = (rank, index).  kRemote = false keeps every update on the own CTA.
template <int kOps, bool kRemote>
__global__ void cluster_kernel(Agg* out, uint32_t slots_per_cta, int64_t updates_per_thread) {
  extern __shared__ __align__(32) unsigned char smem[];
  Agg* t = reinterpret_cast<Agg*>(smem);
  cg::cluster_group cl = cg::this_cluster();
  const unsigned C = cl.num_blocks();
  const unsigned me = cl.block_rank();
  for (uint32_t i = threadIdx.x; i < slots_per_cta; i += blockDim.x) t[i] = Agg{0, 0, INT64_MAX, INT64_MIN};
  cl.sync();
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t total = (uint64_t)slots_per_cta * C;
  for (int64_t k = 0; k < updates_per_thread; ++k) {
    const uint64_t h = mix(tid * 1000003ull + k);
    const uint32_t g = (uint32_t)(((h >> 32) * total) >> 32);  // < total
    const unsigned rank = kRemote ? g % C : me;                 // < C
    const uint32_t idx = g / C;                                 // < slots_per_cta
    Agg* p = cl.map_shared_rank(t, rank) + idx;
    upd<kOps>(p, (int64_t)(h & 0xFFFFFF));
  }
  cl.sync();
  // fold the CTA's slice into out so the work is observable (out has slots_per_cta entries)
  for (uint32_t i = threadIdx.x; i < slots_per_cta; i += blockDim.x) {
    atomicAdd(&out[i].sum, t[i].sum);
    atomicAdd(&out[i].cnt, t[i].cnt);
  }
}

template <typename K>
float time_launch(K launch, int reps) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  launch();
  CK(cudaDeviceSynchronize());
  CK(cudaEventRecord(a));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(b));
  CK(cudaEventSynchronize(b));
  float ms;
  CK(cudaEventElapsedTime(&ms, a, b));
  CK(cudaGetLastError());
  return ms / reps;
}

int main() {
  int sms;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const int64_t updates = 180000000;  // selected rows of the 600M-row query
  // L2 reductions
  {
    Agg* tab;
    const uint32_t slots = 262144;
    CK(cudaMalloc(&tab, sizeof(Agg) * slots));
    CK(cudaMemset(tab, 0, sizeof(Agg) * slots));
    const int threads = 256, blocks = sms * 8;
    const int64_t per = updates / ((int64_t)threads * blocks);
    const double n = (double)per * threads * blocks;
    float ms4 = time_launch([&] { l2_kernel<4><<<blocks, threads>>>(tab, slots, per); }, 3);
    float ms2 = time_launch([&] { l2_kernel<2><<<blocks, threads>>>(tab, slots, per); }, 3);
    printf("L2 RED, %u slots: 4 ops %.3f ms (%.1f G ops/s), 2 ops %.3f ms (%.1f G ops/s)\n", slots, ms4,
           4 * n / ms4 / 1e6, ms2, 2 * n / ms2 / 1e6);
    CK(cudaFree(tab));
  }
  for (int C : {8, 16}) {
    for (uint32_t spc : {6272u, 3200u}) {  // ~196 KB and 100 KB of aggregates per CTA
      const size_t smem = (size_t)spc * sizeof(Agg);
      for (int threads : {512, 1024}) {
        auto kr = cluster_kernel<4, true>;
        CK(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CK(cudaFuncSetAttribute(kr, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        auto kl = cluster_kernel<4, false>;
        CK(cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CK(cudaFuncSetAttribute(kl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        auto k2 = cluster_kernel<2, true>;
        CK(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CK(cudaFuncSetAttribute(k2, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.gridDim = dim3(C);
        int nclusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, (void*)kr, &cfg);
        if (e != cudaSuccess || nclusters == 0) {
          printf("C=%d smem=%zu threads=%d: no active clusters (%s)\n", C, smem, threads, cudaGetErrorString(e));
          cudaGetLastError();
          continue;
        }
        cfg.gridDim = dim3(nclusters * C);
        Agg* out;
        CK(cudaMalloc(&out, sizeof(Agg) * spc));
        CK(cudaMemset(out, 0, sizeof(Agg) * spc));
        const int64_t per = updates / ((int64_t)threads * nclusters * C);
        const double n = (double)per * threads * nclusters * C;
        float msr = time_launch([&] { CK(cudaLaunchKernelEx(&cfg, kr, out, spc, per)); }, 3);
        float msl = time_launch([&] { CK(cudaLaunchKernelEx(&cfg, kl, out, spc, per)); }, 3);
        float ms2 = time_launch([&] { CK(cudaLaunchKernelEx(&cfg, k2, out, spc, per)); }, 3);
        printf("C=%2d smem=%6zu threads=%4d clusters=%2d (%3d SMs): remote 4 ops %.3f ms (%.1f G ops/s) | "
               "local 4 ops %.3f ms (%.1f G ops/s) | remote 2 ops %.3f ms (%.1f G ops/s)\n",
               C, smem, threads, nclusters, nclusters * C, msr, 4 * n / msr / 1e6, msl, 4 * n / msl / 1e6, ms2,
               2 * n / ms2 / 1e6);
        CK(cudaFree(out));
      }
    }
  }
  return 0;
}
