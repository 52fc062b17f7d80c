// k_probe.cu -- rd_probe_mma: the rate of the tensor-core instruction the split path's digit
// products use, measured on this GPU with nothing else in the loop (the ceiling the split GEMM is
// held against).
//
// One CTA per SM; one thread issues tcgen05.mma.kind::f16 (BF16 A and B, FP32 accumulator,
// M = N = 128, K = 16, operands in shared memory as 128-byte swizzled K-major tiles, accumulator
// in tensor memory) back to back, 64 MMAs per commit, and waits (bounded) for each commit before
// the next batch.  The operands are zeros: the rate of the tensor pipe does not depend on them.
// The 8-bit integer kind (tcgen05.mma.kind::i8, int32 accumulation), the other exact digit format,
// does not exist for sm_103a: ptxas refuses it ("Feature '.kind::i8' not supported on .target
// 'sm_103a'"), so INT8 digits are not an option on this GPU.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "rd_internal.cuh"

namespace {

constexpr int PT = 128;             // threads per CTA
constexpr int PTILE = 128 * 128;    // bytes of one operand tile (128 rows of 128 bytes)
constexpr int BATCH = 64;           // MMAs per commit
constexpr unsigned long long PROBE_WAIT_NS = 2000000000ull;

// f32 <- bf16 x bf16, N = 128, M = 128
constexpr uint32_t IDESC_PROBE = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ unsigned long long probe_time() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(PT, 1) probe_mma_kernel(int batches, int* status, unsigned long long* ns) {
  extern __shared__ uint8_t psm_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)psm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;
  uint8_t* sB = sm + PTILE;
  uint64_t* bar = (uint64_t*)(sm + 2 * PTILE);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int t = threadIdx.x;
  for (int e = t; e < 2 * PTILE / 16; e += PT) reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, before the tensor core reads them
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (t == 0) {
    const uint32_t a = smem_addr(sA), b = smem_addr(sB);
    const unsigned long long t0 = probe_time();
    bool ok = true;
    for (int q = 0; q < batches && ok; ++q) {
      for (int i = 0; i < BATCH; ++i) {
        const uint64_t da = desc_sw128(a + (i & 3) * 32), db = desc_sw128(b + (i & 3) * 32);
        const uint32_t acc = (q | i) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(IDESC_PROBE), "r"(acc)
                     : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                   : "memory");
      // wait for this batch (phase q), bounded
      const unsigned long long dl = probe_time() + PROBE_WAIT_NS;
      uint32_t done = 0;
      while (!done) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"((uint32_t)(q & 1))
            : "memory");
        if (!done && probe_time() > dl) {
          ok = false;
          break;
        }
      }
    }
    const unsigned long long t1 = probe_time();
    if (!ok) rd_set_status(status, RD_DEV_TIMEOUT, blockIdx.x);
    atomicMax(ns, t1 - t0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (t < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
  }
}

}  // namespace

extern "C" rd_status rd_probe_mma(int32_t kind, int32_t batches, double* tera_ops, double* seconds) {
  if (!tera_ops || !seconds || (kind != 0 && kind != 1) || batches < 1 || batches > 1000000) {
    rd_record_error("rd_probe_mma: kind 0 (BF16) or 1 (INT8), 1 <= batches <= 1e6, outputs not NULL");
    return RD_ERR_ARG;
  }
  if (kind == 1) {
    rd_record_error("rd_probe_mma: tcgen05.mma.kind::i8 does not exist for sm_103a (ptxas: Feature '.kind::i8' "
                    "not supported on .target 'sm_103a')");
    return RD_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int* status = nullptr;
  unsigned long long* ns = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ns, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(status, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ns, 0, sizeof(unsigned long long));
  // two 16 KiB tiles and the barrier; 128 KiB requested so that no two probe CTAs share an SM
  const int smem = 128 * 1024;
  if (e == cudaSuccess) {
    e = cudaFuncSetAttribute(probe_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) probe_mma_kernel<<<sms, PT, smem>>>(batches, status, ns);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int st[2] = {0, 0};
  unsigned long long t = 0;
  if (e == cudaSuccess) e = cudaMemcpy(st, status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&t, ns, sizeof(t), cudaMemcpyDeviceToHost);
  if (status) cudaFree(status);
  if (ns) cudaFree(ns);
  if (e != cudaSuccess) {
    rd_record_error(std::string("rd_probe_mma: ") + cudaGetErrorString(e));
    return RD_ERR_CUDA;
  }
  if (st[0] != 0) {
    rd_record_error("rd_probe_mma: a bounded wait for the tensor core expired");
    return RD_ERR_TIMEOUT;
  }
  const double ops = (double)sms * batches * BATCH * 2.0 * 128.0 * 128.0 * 16.0;
  *seconds = (double)t * 1e-9;
  *tera_ops = t ? ops / (double)t * 1e-3 : 0.0;
  return RD_OK;
}
