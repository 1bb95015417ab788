// Accuracy of the FP32 pass's own e^x - 1 and square root (quad32.cuh:
// emq::ex_m1, emq::sqrt_nr) against a double-precision host reference and
// against CUDA's expm1f / sqrtf, over dense samples of the ranges the pass
// uses.  Prints, per function, its name, its largest error in ulps against
// the reference, the CUDA call's on the same inputs, and the sample count;
// built and run by tests/test_gpu_fastmath.py.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "quad32.cuh"

__global__ void eval(int n, const float *x, float *own_e, float *lib_e, float *own_s, float *lib_s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    own_e[i] = emq::ex_m1(x[i]);
    lib_e[i] = expm1f(x[i]);
    const float a = fabsf(x[i]);
    own_s[i] = emq::sqrt_nr(a);
    lib_s[i] = sqrtf(a);
}

// distance in units in the last place of the FP32 rounding of ref
static double ulps(float y, double ref)
{
    const float rf = (float)ref;
    if (rf == 0.f) return y == 0.f ? 0.0 : 1e30;
    int e;
    std::frexp(std::fabs((double)rf), &e);
    const double ulp = std::ldexp(1.0, std::max(e - 24, -149));
    return std::fabs((double)y - ref) / ulp;
}

int main()
{
    std::vector<float> x;
    for (int i = 0; i < 1 << 20; ++i) x.push_back(-10.f + 80.5f * (float)i / (float)(1 << 20));   // [-10, 70.5]
    for (int i = 0; i < 1 << 18; ++i) x.push_back(std::ldexp(1.f, -60) * std::pow(2.f, 60.f * i / (1 << 18)));
    for (int i = 0; i < 1 << 16; ++i) x.push_back(-std::ldexp(1.f, -40) * std::pow(2.f, 40.f * i / (1 << 16)));
    for (int i = 1; i < 1 << 12; ++i) x.push_back(std::ldexp((float)i, -149));   // subnormals
    x.push_back(0.f);
    const int n = (int)x.size();
    float *d[5];
    for (auto &p : d)
        if (cudaMalloc(&p, n * sizeof(float)) != cudaSuccess) return 1;
    cudaMemcpy(d[0], x.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    eval<<<(n + 255) / 256, 256>>>(n, d[0], d[1], d[2], d[3], d[4]);
    std::vector<float> oe(n), le(n), os(n), ls(n);
    cudaMemcpy(oe.data(), d[1], n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(le.data(), d[2], n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(os.data(), d[3], n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(ls.data(), d[4], n * sizeof(float), cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) return 2;
    double me = 0, mel = 0, ms = 0, msl = 0;
    for (int i = 0; i < n; ++i) {
        const double re = std::expm1((double)x[i]);
        me = std::max(me, ulps(oe[i], re));
        mel = std::max(mel, ulps(le[i], re));
        const double rs = std::sqrt(std::fabs((double)x[i]));
        ms = std::max(ms, ulps(os[i], rs));
        msl = std::max(msl, ulps(ls[i], rs));
    }
    std::printf("ex_m1 %.3f %.3f %d\n", me, mel, n);
    std::printf("sqrt_nr %.3f %.3f %d\n", ms, msl, n);
    return 0;
}
