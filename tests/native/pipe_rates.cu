// Issue-rate microbenchmark of the arithmetic the two precision paths rely
// on: FP64 add and fma, f32 <-> f64 conversion, FP32 fma, and 32-bit integer
// add/logic, in thread-operations per clock per SM.  Four independent chains
// per thread, 8 blocks of 256 threads per SM; every thread writes one result
// (index < blocks * threads, the allocated size).  Prints one line per
// operation: "<name> <ops per clock per SM>".
#include <cuda_runtime.h>
#include <stdio.h>

template <int OP>
__global__ void chains(double *outd, float *outf, unsigned *outu, int iters, double seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d0 = seed + i, d1 = seed - i, d2 = 0.5 * seed + i, d3 = 0.25 * seed - i;
    float f0 = (float)d0, f1 = (float)d1, f2 = (float)d2, f3 = (float)d3;
    unsigned u0 = i, u1 = i * 3u, u2 = i * 5u, u3 = i * 7u;
    for (int k = 0; k < iters; ++k) {
        if (OP == 0) { d0 += 1.0000001; d1 += 0.9999999; d2 += 1.0000003; d3 += 0.9999997; }
        if (OP == 1) {
            d0 = fma(d0, 0.9999999, 1e-7); d1 = fma(d1, 0.9999998, 2e-7);
            d2 = fma(d2, 0.9999997, 3e-7); d3 = fma(d3, 0.9999996, 4e-7);
        }
        if (OP == 2) {  // two conversions per chain step
            f0 = (float)((double)f0 + 1e-9); f1 = (float)((double)f1 + 2e-9);
            f2 = (float)((double)f2 + 3e-9); f3 = (float)((double)f3 + 4e-9);
        }
        if (OP == 3) {
            f0 = fmaf(f0, 0.9999999f, 1e-7f); f1 = fmaf(f1, 0.9999998f, 2e-7f);
            f2 = fmaf(f2, 0.9999997f, 3e-7f); f3 = fmaf(f3, 0.9999996f, 4e-7f);
        }
        if (OP == 4) {
            u0 = (u0 + 0x9E3779B9u) ^ (u0 >> 3); u1 = (u1 + 0x7F4A7C15u) ^ (u1 >> 5);
            u2 = (u2 + 0x94D049BBu) ^ (u2 >> 7); u3 = (u3 + 0xBF58476Du) ^ (u3 >> 11);
        }
    }
    outd[i] = d0 + d1 + d2 + d3;
    outf[i] = f0 + f1 + f2 + f3;
    outu[i] = u0 ^ u1 ^ u2 ^ u3;
}

int main()
{
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const int threads = 256, blocks = sms * 8, n = blocks * threads, iters = 2048;
    double *d = nullptr;
    float *f = nullptr;
    unsigned *u = nullptr;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&u, n * sizeof(unsigned)) != cudaSuccess)
        return 1;
    const char *names[] = {"dadd", "dfma", "cvt_f32_f64", "ffma", "int_add_xor_shift"};
    // operations per chain step: 4 chains x (1 op, 1 op, 2 conversions, 1 op, 3 int ops)
    const double per_iter[] = {4, 4, 8, 4, 12};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int op = 0; op < 5; ++op) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // the second launch is timed
            cudaEventRecord(a);
            switch (op) {
            case 0: chains<0><<<blocks, threads>>>(d, f, u, iters, 1.5); break;
            case 1: chains<1><<<blocks, threads>>>(d, f, u, iters, 1.5); break;
            case 2: chains<2><<<blocks, threads>>>(d, f, u, iters, 1.5); break;
            case 3: chains<3><<<blocks, threads>>>(d, f, u, iters, 1.5); break;
            default: chains<4><<<blocks, threads>>>(d, f, u, iters, 1.5); break;
            }
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
        }
        const double ops = (double)n * iters * per_iter[op];
        const double per_clk_sm = ops / (ms * 1e-3) / sms / (clk_khz * 1e3);
        printf("%s %.3f\n", names[op], per_clk_sm);
    }
    printf("status %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
