// selfcheck.cu -- device check of the paired FP32 reciprocal (Pair<float>::rcp)
// that the tiled and batched kernels use for u' = m' / rho' (Eq. (5)), and a
// measurement of the device's paired-FP32 FMA rate (the arithmetic ceiling the
// D3Q19 step is checked against beside the memory roofline).

#include "step_tiled.cuh"

namespace maclab {

namespace {

// x_i = lo (hi / lo)^(i / (n - 1)); the largest |rcp(x) x - 1| over all points,
// as the bit pattern of a non-negative double (ordered like unsigned integers).
__global__ void rcp_check_k(double lo, double ratio, int n, unsigned long long* worst) {
  const int i0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= n) return;
  const int i1 = i0 + 1 < n ? i0 + 1 : i0;
  const double den = n > 1 ? (double)(n - 1) : 1.0;
  const float x0 = (float)(lo * pow(ratio, i0 / den));
  const float x1 = (float)(lo * pow(ratio, i1 / den));
  const float2 r = Pair<float>::rcp(make_float2(x0, x1));
  const double e0 = fabs((double)r.x * (double)x0 - 1.0);
  const double e1 = fabs((double)r.y * (double)x1 - 1.0);
  const double e = e0 > e1 ? e0 : e1;
  atomicMax(worst, (unsigned long long)__double_as_longlong(e));
}

// kChains independent chains x <- x a + b per thread on float2 lanes (one
// paired FMA instruction = two FMAs); a < 1 and b > 0 keep x near b / (1 - a).
constexpr int kChains = 8;
__global__ void fp32_peak_k(int iters, float a, float b, float2* sink) {
  float2 x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2(1e-7f * threadIdx.x + k, 0.5f * k);
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], A, B);
  }
  float2 s = x[0];
#pragma unroll
  for (int k = 1; k < kChains; ++k) s = __fadd2_rn(s, x[k]);
  if (s.x == -1.0f) sink[threadIdx.x] = s;  // never true: keeps the chains live
}

}  // namespace

cudaError_t launch_fp32_peak(int blocks, int threads, int iters, float2* sink, cudaStream_t st,
                             double* flops) {
  fp32_peak_k<<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-6f, sink);
  *flops = (double)blocks * threads * iters * kChains * 4.0;
  return cudaGetLastError();
}

cudaError_t launch_check_reciprocal(float lo, float hi, int n, unsigned long long* d_worst,
                                    cudaStream_t st) {
  const int pairs = (n + 1) / 2;
  const int threads = 256;
  rcp_check_k<<<(pairs + threads - 1) / threads, threads, 0, st>>>((double)lo, (double)hi / (double)lo, n,
                                                                   d_worst);
  return cudaGetLastError();
}

}  // namespace maclab
