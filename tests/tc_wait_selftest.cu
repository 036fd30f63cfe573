// Test kernel for the bounded mbarrier wait of the tensor-core z solve (tc_ptx.cuh): a wait
// on a barrier that nothing arrives at must give up after its limit and let the kernel
// return normally, and a wait on a completed phase must succeed.  Built by the test that
// loads it; not part of the library.
#include <cuda_runtime.h>

#include "../paper_2104_00350_gb300/csrc/tc_ptx.cuh"

__global__ void k_wait(int* out, unsigned long long limit_ns, int arrive) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ibpf::tc::mbar_init(&bar, 1);
    ibpf::tc::mbar_init_fence();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ibpf::tc::smem_u32(&bar)) : "memory");
  const bool ok = ibpf::tc::mbar_wait(&bar, 0, limit_ns);
  if (threadIdx.x == 0) out[0] = ok ? 1 : 2;
}

// result: 1 the wait saw the phase complete, 2 it gave up; returns the CUDA error code
extern "C" int tc_wait_selftest(unsigned long long limit_ns, int arrive, int* result) {
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e != cudaSuccess) return (int)e;
  cudaMemset(d, 0, sizeof(int));
  k_wait<<<1, 32>>>(d, limit_ns, arrive);
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(result, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return (int)e;
}
