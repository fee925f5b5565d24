// k_mg_f32.cu -- FP32 instantiations of the multigrid kernels and the
// shared FP64 sum.
#define BTMG_MG_DEFINE_COMMON
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
INST_TC(float, float)
INST_C(float)
template cudaError_t launch_scale_to<float>(const double*, float*, double, size_t, cudaStream_t);
template cudaError_t launch_refine_update<float>(double*, const float*, double, size_t, cudaStream_t);
template cudaError_t launch_learn_update<float, float>(float*, const float*, size_t, float*, const float*, size_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_learn_dot<float>(const float*, const float*, const Dir<float>*, int, int, int, double, double*, int, double*, cudaStream_t);
template cudaError_t launch_learn_build<float, float>(float*, float*, const float*, const float*, const float*, const Dir<float>*, int, int, int, int, int, double, double, double, cudaStream_t);
template cudaError_t launch_learn_features<float>(const float*, int, const float*, const float*, const float*, const float*, double, int, int, int, int, int, double*, double*, float*, float*, cudaStream_t);
template cudaError_t launch_dphi_norm<float>(const float*, int, const float*, int, double*, int, double*, cudaStream_t);
}  // namespace btmg
