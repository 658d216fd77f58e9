// Explicit instantiation of the solver entry points for the double element type.
#include "solver_impl.cuh"

namespace eot {
template void run_marginals<double>(eot_handle, const eot_problem*, const double*, const double*, double,
                                double*, double*, double*, double*, double*, cudaStream_t);
template void run_value<double>(eot_handle, const eot_problem*, const double*, const double*, double, double*,
                            cudaStream_t);
template void run_hvp<double>(eot_handle, const eot_problem*, const double*, const double*, double, double,
                          const double*, const double*, double*, double*, double*, double*, cudaStream_t);
template void run_newton<double>(eot_handle, const eot_problem*, const double*, const double*, double,
                             const double*, double, double, int, double*, double*, double*, int*, bool,
                             cudaStream_t);
template void run_solve<double>(eot_handle, const eot_problem*, const eot_params*, double*, double*,
                            eot_stats*, cudaStream_t);
template void run_backward_dense<double>(eot_handle, const eot_problem*, const double*, const double*,
                                     double, double, const double*, float*, cudaStream_t);
template double run_sweep_bench<double>(eot_handle, const eot_problem*, const double*, const double*,
                                    double, int, int, void*, size_t, cudaStream_t);
template void run_backward_points<double>(eot_handle, const eot_problem*, const double*, const double*,
                                      double, double, const double*, float*, float*, cudaStream_t);
template void run_round<double>(eot_handle, const eot_problem*, const double*, const double*, double, double*,
                            double*, double*, double*, double*, double*, cudaStream_t);
}  // namespace eot
