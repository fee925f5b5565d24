// k_mg_f64.cu -- FP64 instantiations of the multigrid kernels.
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
INST_TC(double, double)
INST_C(double)
template cudaError_t launch_scale_to<double>(const double*, double*, double, size_t, cudaStream_t);
template cudaError_t launch_refine_update<double>(double*, const double*, double, size_t, cudaStream_t);
template cudaError_t launch_learn_update<double, double>(double*, const double*, size_t, double*, const double*, size_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_learn_dot<double>(const double*, const double*, const Dir<double>*, int, int, int, double, double*, int, double*, cudaStream_t);
template cudaError_t launch_learn_build<double, double>(double*, double*, const float*, const double*, const double*, const Dir<double>*, int, int, int, int, int, double, double, double, cudaStream_t);
template cudaError_t launch_learn_features<double>(const double*, int, const double*, const double*, const double*, const double*, double, int, int, int, int, int, double*, double*, float*, float*, cudaStream_t);
template cudaError_t launch_dphi_norm<double>(const double*, int, const double*, int, double*, int, double*, cudaStream_t);
}  // namespace btmg
