// k_scale.cu -- multiplies a batch of complex elements by a real factor: the
// optional normalisation of an execute's outputs (fftb_plan_set_scale). The
// transform stages stay unscaled as the paper defines them (Sec. 2.1, 2.2);
// this runs after them on the output ranges only.
#include "kernels.cuh"

namespace fftb {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_scale(typename cplx<T>::type* data, int64_t n, T s) {
  pdl_launch_dependents();
  pdl_wait();  // the producing stage has completed
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    typename cplx<T>::type v = data[i];
    v.x *= s;
    v.y *= s;
    data[i] = v;
  }
}

}  // namespace

cudaError_t launch_scale(int csize, void* data, int64_t n, double s, const Launch& L, int sms) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  const dim3 grid((unsigned)std::min<int64_t>(want, (int64_t)sms * 8));
  if (csize == 16) return launch_k(k_scale<double>, grid, 256, 0, L, static_cast<double2*>(data), n, s);
  return launch_k(k_scale<float>, grid, 256, 0, L, static_cast<float2*>(data), n, (float)s);
}

}  // namespace fftb
