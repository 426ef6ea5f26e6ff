// probe_rates.cu -- unit-rate microbenchmarks for the roofline denominators: FP32 FMA (scalar and packed
// f32x2, with and without a negated addend), MUFU ex2 / sin, FP64 DFMA; and the absolute error of
// sin/cos.approx against FP64, with and without the splats' argument reduction
// (CUDA events; every access in bounds, no waits).  Build: nvcc -O3 -gencode arch=compute_103a,code=sm_103a probe_rates.cu
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s @%d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
constexpr int ITERS=4096;
__global__ void k_fma(float* out, float a, float b){
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<ITERS;i++){ x0=fmaf(x0,a,b); x1=fmaf(x1,a,b); x2=fmaf(x2,a,b); x3=fmaf(x3,a,b);
    x4=fmaf(x4,a,b); x5=fmaf(x5,a,b); x6=fmaf(x6,a,b); x7=fmaf(x7,a,b);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
// x = -x * a + b: the negated addend shows whether the sign folds into the instruction
__global__ void k_fma_neg(float* out, float a, float b){
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<ITERS;i++){ x0=fmaf(a,b,-x0); x1=fmaf(a,b,-x1); x2=fmaf(a,b,-x2); x3=fmaf(a,b,-x3);
    x4=fmaf(a,b,-x4); x5=fmaf(a,b,-x5); x6=fmaf(a,b,-x6); x7=fmaf(a,b,-x7);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
template <bool NEG>
__global__ void k_ffma2(float* out, float a, float b){
  const float2 a2=make_float2(a,a), b2=make_float2(b,b);
  float2 x[8];
  for(int j=0;j<8;j++) x[j]=make_float2(threadIdx.x+j, threadIdx.x+j+0.5f);
  for(int i=0;i<ITERS;i++){
#pragma unroll
    for(int j=0;j<8;j++) x[j] = NEG ? __ffma2_rn(a2, b2, make_float2(-x[j].x, -x[j].y)) : __ffma2_rn(x[j], a2, b2);
  }
  float s=0.f;
  for(int j=0;j<8;j++) s+=x[j].x+x[j].y;
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__device__ __forceinline__ float ex2(float x){float y; asm volatile("ex2.approx.ftz.f32 %0, %1;":"=f"(y):"f"(x)); return y;}
__device__ __forceinline__ float sn(float x){float y; asm volatile("sin.approx.ftz.f32 %0, %1;":"=f"(y):"f"(x)); return y;}
__global__ void k_ex2(float* out, float a){
  float x0=threadIdx.x*1e-3f, x1=x0+.1f, x2=x0+.2f, x3=x0+.3f, x4=x0+.4f, x5=x0+.5f, x6=x0+.6f, x7=x0+.7f;
  for(int i=0;i<ITERS;i++){ x0=ex2(x0)*a; x1=ex2(x1)*a; x2=ex2(x2)*a; x3=ex2(x3)*a; x4=ex2(x4)*a; x5=ex2(x5)*a; x6=ex2(x6)*a; x7=ex2(x7)*a;}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_ex2only(float* out){
  float x0=threadIdx.x*1e-3f, x1=x0+.1f, x2=x0+.2f, x3=x0+.3f, x4=x0+.4f, x5=x0+.5f, x6=x0+.6f, x7=x0+.7f;
  for(int i=0;i<ITERS;i++){ x0=ex2(x0); x1=ex2(x1); x2=ex2(x2); x3=ex2(x3); x4=ex2(x4); x5=ex2(x5); x6=ex2(x6); x7=ex2(x7);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_sin(float* out){
  float x0=threadIdx.x*1e-3f, x1=x0+.1f, x2=x0+.2f, x3=x0+.3f, x4=x0+.4f, x5=x0+.5f, x6=x0+.6f, x7=x0+.7f;
  for(int i=0;i<ITERS;i++){ x0=sn(x0); x1=sn(x1); x2=sn(x2); x3=sn(x3); x4=sn(x4); x5=sn(x5); x6=sn(x6); x7=sn(x7);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_dfma(double* out, double a, double b){
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3;
  for(int i=0;i<ITERS/8;i++){ x0=fma(x0,a,b); x1=fma(x1,a,b); x2=fma(x2,a,b); x3=fma(x3,a,b);}
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3;
}
// accuracy of sin/cos.approx against FP64 on [-X, X]: unreduced arguments, and after the FP32
// reduction t - 2 pi round(t / 2 pi) (+-1.5 2^23 rounding) that the splats use
__device__ __forceinline__ float cs_(float x){float y; asm("cos.approx.ftz.f32 %0, %1;":"=f"(y):"f"(x)); return y;}
__device__ __forceinline__ float sn_(float x){float y; asm("sin.approx.ftz.f32 %0, %1;":"=f"(y):"f"(x)); return y;}
__global__ void k_sin_err(float X, int n, unsigned long long* err_raw, unsigned long long* err_red){
  int i = blockIdx.x*blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = -X + (2.0f*X) * ((float)i + 0.5f) / (float)n;
  const double xs = (double)x;
  const double ts = sin(xs), tc = cos(xs);
  const float kr = __fadd_rn(fmaf(x, 0.15915494309189535f, 12582912.0f), -12582912.0f);
  const float r = fmaf(kr, -6.28318530717958647692f, x);
  const double e1 = fmax(fabs((double)sn_(x) - ts), fabs((double)cs_(x) - tc));
  const double e2 = fmax(fabs((double)sn_(r) - ts), fabs((double)cs_(r) - tc));
  atomicMax(err_raw, (unsigned long long)__double_as_longlong(e1));  // non-negative doubles order as integers
  atomicMax(err_red, (unsigned long long)__double_as_longlong(e2));
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  int clk=0, memclk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0); cudaDeviceGetAttribute(&memclk, cudaDevAttrMemoryClockRate, 0);
  printf("{\"name\":\"%s\",\"sms\":%d,\"cc\":\"%d.%d\",\"clock_khz\":%d,\"smem_optin\":%zu,\"regs_per_sm\":%d,\"l2\":%d}\n", p.name, p.multiProcessorCount, p.major,p.minor, clk, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor, p.l2CacheSize);
  int blocks=p.multiProcessorCount*8, threads=256; size_t n=(size_t)blocks*threads;
  float* o; double* od; CK(cudaMalloc(&o,n*4)); CK(cudaMalloc(&od,n*8));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int rep=0;rep<3;rep++){
    k_fma<<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e0)); k_fma<<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double fma_rate = (double)n*ITERS*8/(ms*1e-3); printf("fp32 fma/s %.4g  per SM per clk(at %d kHz) %.2f\n", fma_rate, clk, fma_rate/p.multiProcessorCount/(clk*1e3));
    k_fma_neg<<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e0)); k_fma_neg<<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    fma_rate = (double)n*ITERS*8/(ms*1e-3); printf("fp32 fma (negated addend) /s %.4g per SM per clk %.2f\n", fma_rate, fma_rate/p.multiProcessorCount/(clk*1e3));
    k_ffma2<false><<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e0)); k_ffma2<false><<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    fma_rate = (double)n*ITERS*8/(ms*1e-3); printf("fp32x2 ffma2 instr/s %.4g per SM per clk %.2f (lane-FMAs x2)\n", fma_rate, fma_rate/p.multiProcessorCount/(clk*1e3));
    k_ffma2<true><<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e0)); k_ffma2<true><<<blocks,threads>>>(o,0.999f,0.001f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    fma_rate = (double)n*ITERS*8/(ms*1e-3); printf("fp32x2 ffma2 (negated addend) instr/s %.4g per SM per clk %.2f\n", fma_rate, fma_rate/p.multiProcessorCount/(clk*1e3));
    k_ex2<<<blocks,threads>>>(o,0.5f); CK(cudaEventRecord(e0)); k_ex2<<<blocks,threads>>>(o,0.5f); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double ex2_rate=(double)n*ITERS*8/(ms*1e-3); printf("ex2+fmul pairs/s %.4g per SM per clk %.2f\n", ex2_rate, ex2_rate/p.multiProcessorCount/(clk*1e3));
    k_ex2only<<<blocks,threads>>>(o); CK(cudaEventRecord(e0)); k_ex2only<<<blocks,threads>>>(o); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    ex2_rate=(double)n*ITERS*8/(ms*1e-3); printf("ex2 only /s %.4g per SM per clk %.2f\n", ex2_rate, ex2_rate/p.multiProcessorCount/(clk*1e3));
    k_sin<<<blocks,threads>>>(o); CK(cudaEventRecord(e0)); k_sin<<<blocks,threads>>>(o); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double sin_rate=(double)n*ITERS*8/(ms*1e-3); printf("sin.approx /s %.4g per SM per clk %.2f\n", sin_rate, sin_rate/p.multiProcessorCount/(clk*1e3));
    k_dfma<<<blocks,threads>>>(od,0.999,0.001); CK(cudaEventRecord(e0)); k_dfma<<<blocks,threads>>>(od,0.999,0.001); CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double d_rate=(double)n*(ITERS/8)*4/(ms*1e-3); printf("fp64 dfma/s %.4g per SM per clk %.3f\n", d_rate, d_rate/p.multiProcessorCount/(clk*1e3));
  }
  unsigned long long *eb; CK(cudaMalloc(&eb, 16));
  const float Xs[] = {3.14159265f, 31.4159265f, 314.159265f, 1000.0f};
  for (float X : Xs) {
    CK(cudaMemset(eb, 0, 16));
    const int n = 1 << 24;
    k_sin_err<<<n / 256, 256>>>(X, n, eb, eb + 1);
    unsigned long long h[2]; CK(cudaMemcpy(h, eb, 16, cudaMemcpyDeviceToHost));
    double e[2]; memcpy(e, h, 16);
    printf("sin/cos.approx max abs error on [-%g, %g]: unreduced %.3g, reduced %.3g\n", X, X, e[0], e[1]);
  }
  CK(cudaDeviceSynchronize()); printf("ok\n"); return 0;
}
