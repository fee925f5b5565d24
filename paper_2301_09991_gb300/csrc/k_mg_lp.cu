// k_mg_lp.cu -- BF16 / FP16 storage instantiations (FP32 compute).
#include "k_mg_impl.cuh"

namespace btmg {
#define INST_TC(T, C)                                                                                  \
  template cudaError_t launch_upwind<T, C>(const UpArgs<T, C>&, int, int, cudaStream_t);                \
  template cudaError_t launch_phi_partial<T, C>(const T*, C*, const Dir<C>*, int, int, int, int, int, cudaStream_t);
#define INST_C(C)                                                                                          \
  template cudaError_t launch_restrict<C>(const C*, C*, const C*, int, int, int, int, int, int, int, int, int, int, \
                                          int, int, cudaStream_t);                                         \
  template cudaError_t launch_prolong<C>(const C*, C*, int, int, int, int, int, int, int, int, int, int, int, int, \
                                         cudaStream_t);                                                    \
  template cudaError_t launch_source<C>(const C*, const C*, const C*, int, int, int, int, C*, C*, double*, int, \
                                        cudaStream_t);                                                     \
  template cudaError_t launch_phi_sum<C>(const C*, int, int, C*, cudaStream_t);
INST_TC(__nv_bfloat16, float)
INST_TC(__half, float)
template cudaError_t launch_refine_update<__nv_bfloat16>(double*, const __nv_bfloat16*, double, size_t, cudaStream_t);
template cudaError_t launch_refine_update<__half>(double*, const __half*, double, size_t, cudaStream_t);
template cudaError_t launch_learn_update<__nv_bfloat16, float>(__nv_bfloat16*, const __nv_bfloat16*, size_t, float*, const float*, size_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_learn_update<__half, float>(__half*, const __half*, size_t, float*, const float*, size_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_learn_build<__nv_bfloat16, float>(__nv_bfloat16*, float*, const float*, const float*, const float*, const Dir<float>*, int, int, int, int, int, double, double, double, cudaStream_t);
template cudaError_t launch_learn_build<__half, float>(__half*, float*, const float*, const float*, const float*, const Dir<float>*, int, int, int, int, int, double, double, double, cudaStream_t);
}  // namespace btmg
