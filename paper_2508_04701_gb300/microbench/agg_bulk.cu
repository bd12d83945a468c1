// Microbenchmark: 180M aggregate updates into random 32-byte slots of a 262144-slot table in
// L2, two ways:
//   RED4 : four fire-and-forget reductions (add sum, add count, min, max) -- the fused probe's
//   BULK2: two 16-byte bulk reductions from shared memory (cp.reduce.async.bulk, the TMA
//          unit): add.u64 on {sum, count} and min.s64 on {min, ~max} (MAX kept as the
//          bitwise complement, which reverses the order, so one MIN serves both)
// with 1, 2 or 4 staging buffers per thread, and checks that both give the same table.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o agg_bulk agg_bulk.cu && ./agg_bulk
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e)); exit(1); } } while (0)

__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct __align__(32) Agg { unsigned long long sum, cnt; long long mn, mx; };  // BULK2: mx holds ~max

__global__ void red4_kernel(Agg* tab, uint32_t slots, int64_t per) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (int64_t k = 0; k < per; ++k) {
    const uint64_t h = mix(tid * 1000003ull + k);
    const uint32_t s = (uint32_t)(((h >> 32) * (uint64_t)slots) >> 32);
    const long long v = (long long)(h & 0xFFFFFF) - 0x800000;
    atomicAdd(&tab[s].sum, (unsigned long long)v);
    atomicAdd(&tab[s].cnt, 1ull);
    atomicMin(&tab[s].mn, v);
    atomicMax(&tab[s].mx, v);
  }
}

template <int kBuf>
__global__ void bulk2_kernel(Agg* tab, uint32_t slots, int64_t per) {
  extern __shared__ __align__(16) unsigned long long stage[];  // [kBuf][blockDim][4]
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (int64_t k = 0; k < per; ++k) {
    const int b = (int)(k % kBuf);
    unsigned long long* my = stage + ((size_t)b * blockDim.x + threadIdx.x) * 4;
    // the bulk groups older than the kBuf-1 newest have finished reading their staging
    if (kBuf == 1) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    else asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kBuf - 1) : "memory");
    const uint64_t h = mix(tid * 1000003ull + k);
    const uint32_t s = (uint32_t)(((h >> 32) * (uint64_t)slots) >> 32);
    const long long v = (long long)(h & 0xFFFFFF) - 0x800000;
    my[0] = (unsigned long long)v;
    my[1] = 1ull;
    my[2] = (unsigned long long)v;
    my[3] = (unsigned long long)~v;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(my);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], 16;"
                 :: "l"(&tab[s].sum), "r"(src) : "memory");
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.min.s64 [%0], [%1], 16;"
                 :: "l"(&tab[s].mn), "r"(src + 16) : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
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

__global__ void init_kernel(Agg* t, uint32_t slots, bool negmax) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x)
    t[i] = Agg{0, 0, INT64_MAX, negmax ? INT64_MAX : INT64_MIN};
}

int main() {
  int sms;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const uint32_t slots = 262144;
  const int64_t updates = 180000000;
  Agg *ta, *tb;
  CK(cudaMalloc(&ta, sizeof(Agg) * slots));
  CK(cudaMalloc(&tb, sizeof(Agg) * slots));
  {
    const int threads = 256, blocks = sms * 8;
    const int64_t per = updates / ((int64_t)threads * blocks);
    const double n = (double)per * threads * blocks;
    float ms = time_launch([&] { red4_kernel<<<blocks, threads>>>(ta, slots, per); }, 3);
    printf("RED4  %4d x %4d: %.3f ms  %.1f G updates/s\n", blocks, threads, ms, n / ms / 1e6);
  }
  for (int threads : {128, 256, 512}) {
    for (int bps : {4, 8}) {
      const int blocks = sms * bps;
      const int64_t per = updates / ((int64_t)threads * blocks);
      const double n = (double)per * threads * blocks;
      const size_t smem1 = (size_t)threads * 32, smem2 = 2 * smem1, smem4 = 4 * smem1;
      CK(cudaFuncSetAttribute(bulk2_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4));
      float m1 = time_launch([&] { bulk2_kernel<1><<<blocks, threads, smem1>>>(tb, slots, per); }, 3);
      float m2 = time_launch([&] { bulk2_kernel<2><<<blocks, threads, smem2>>>(tb, slots, per); }, 3);
      float m4 = time_launch([&] { bulk2_kernel<4><<<blocks, threads, smem4>>>(tb, slots, per); }, 3);
      printf("BULK2 %4d x %4d: buf1 %.3f ms %.1f G/s | buf2 %.3f ms %.1f G/s | buf4 %.3f ms %.1f G/s\n", blocks,
             threads, m1, n / m1 / 1e6, m2, n / m2 / 1e6, m4, n / m4 / 1e6);
    }
  }
  // equality check on one run each from identity
  {
    const int threads = 256, blocks = sms * 8;
    const int64_t per = 1000;
    init_kernel<<<1024, 256>>>(ta, slots, false);
    init_kernel<<<1024, 256>>>(tb, slots, true);
    red4_kernel<<<blocks, threads>>>(ta, slots, per);
    bulk2_kernel<2><<<blocks, threads, threads * 64>>>(tb, slots, per);
    CK(cudaDeviceSynchronize());
    std::vector<Agg> a(slots), b(slots);
    CK(cudaMemcpy(a.data(), ta, sizeof(Agg) * slots, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(b.data(), tb, sizeof(Agg) * slots, cudaMemcpyDeviceToHost));
    long bad = 0;
    for (uint32_t i = 0; i < slots; ++i)
      if (a[i].sum != b[i].sum || a[i].cnt != b[i].cnt || a[i].mn != b[i].mn || a[i].mx != ~b[i].mx) ++bad;
    printf("equality check: %ld of %u slots differ\n", bad, slots);
  }
  return 0;
}
