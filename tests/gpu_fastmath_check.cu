// Accuracy of the FP32 pass's own e^x - 1 and square root (quad32.cuh:
// emq::ex_m1, emq::sqrt_nr) against a double-precision host reference and
// against CUDA's expm1f / sqrtf, over dense samples of the ranges the pass
// uses.  Prints, per function, its name, its largest error in ulps against
// the reference, the CUDA call's on the same inputs, and the sample count.
// Then the integer double -> float-float split (split.cuh: em::split_df)
// against the conversions (float)x and (float)(x - (double)(float)x) on the
// host: its name, the number of results that differ in any bit, and the
// sample count.  Built and run by tests/test_gpu_fastmath.py.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "quad32.cuh"
#include "split.cuh"

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

__global__ void split(int n, const double *x, float *hi, float *lo, float *h32, double *w64, float *rn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    em::split_df(x[i], hi[i], lo[i]);
    const double a = fabs(x[i]);
    const bool in = a >= 0x1p-100 && a < 0x1p100;   // the range of f32_of
    h32[i] = in ? em::f32_of(x[i]) : 0.f;
    w64[i] = in ? em::f64_of(hi[i]) : 0.0;
    rn[i] = em::f32_rn(x[i]);
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

    // the split: random significands over binades 2^-90 .. 2^60 (both sides
    // of the 2^-60 switch), exact ties of the rounding with even and odd
    // kept parts, the carry to the next binade, and zeros
    std::vector<double> xd;
    unsigned long long st = 0x9e3779b97f4a7c15ull;
    auto next = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return st;
    };
    for (int i = 0; i < 1 << 20; ++i) {
        const unsigned long long m = next() & 0xfffffffffffffull;
        const int e = 1023 - 90 + (int)(next() % 151);
        const unsigned long long s = next() & 1ull;
        const unsigned long long u = (s << 63) | ((unsigned long long)e << 52) | m;
        double v;
        std::memcpy(&v, &u, 8);
        xd.push_back(v);
        unsigned long long t = (u & ~0x1fffffffull) | 0x10000000ull;   // a tie
        std::memcpy(&v, &t, 8);
        xd.push_back(v);
        t = u | 0xfffffe0000000ull | 0x1fffffffull;                   // carry to the next binade
        std::memcpy(&v, &t, 8);
        xd.push_back(v);
    }
    xd.push_back(0.0);
    xd.push_back(-0.0);
    const int nd = (int)xd.size();
    double *dx, *dw;
    float *dh, *dl, *d32, *drn;
    if (cudaMalloc(&dx, nd * sizeof(double)) != cudaSuccess || cudaMalloc(&dh, nd * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dl, nd * sizeof(float)) != cudaSuccess || cudaMalloc(&d32, nd * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dw, nd * sizeof(double)) != cudaSuccess || cudaMalloc(&drn, nd * sizeof(float)) != cudaSuccess)
        return 3;
    cudaMemcpy(dx, xd.data(), nd * sizeof(double), cudaMemcpyHostToDevice);
    split<<<(nd + 255) / 256, 256>>>(nd, dx, dh, dl, d32, dw, drn);
    std::vector<float> hh(nd), hl(nd), h32(nd), hrn(nd);
    std::vector<double> w64(nd);
    cudaMemcpy(hh.data(), dh, nd * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(hl.data(), dl, nd * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(h32.data(), d32, nd * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(w64.data(), dw, nd * sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemcpy(hrn.data(), drn, nd * sizeof(float), cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) return 4;
    int bad = 0, bad2 = 0, n2 = 0;
    for (int i = 0; i < nd; ++i) {
        const float h = (float)xd[i], l = (float)(xd[i] - (double)h);
        bad += std::memcmp(&h, &hh[i], 4) != 0 || std::memcmp(&l, &hl[i], 4) != 0 || std::memcmp(&h, &hrn[i], 4) != 0;
        const double a = std::fabs(xd[i]);
        if (a >= 0x1p-100 && a < 0x1p100) {
            const double wd = (double)h;
            bad2 += std::memcmp(&h, &h32[i], 4) != 0 || std::memcmp(&wd, &w64[i], 8) != 0;
            ++n2;
        }
    }
    std::printf("split_df %d 0 %d\n", bad, nd);
    std::printf("f32_f64_of %d 0 %d\n", bad2, n2);
    return 0;
}
