// k_split.cu -- split-precision path (BF16 slice products on the tensor cores).  Placeholder
// until the tcgen05 kernels land: the mode reports RD_ERR_UNSUPPORTED.
#include "rd_internal.cuh"

rd_status rd_split_prepare(rd_ctx* h) {
  h->err = "split precision is not built yet";
  return RD_ERR_UNSUPPORTED;
}
void rd_split_release(rd_ctx*) {}
cudaError_t rd_lu_split(rd_ctx*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t rd_trtri_split(rd_ctx*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t rd_trmm_decode_split(rd_ctx*, int32_t*, double*, cudaStream_t) { return cudaErrorNotSupported; }
