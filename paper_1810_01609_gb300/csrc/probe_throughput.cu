// Throughput probe of the ALU rooflines used for the FP64 / FP32 paths (not part of
// libmdwf): FP64 FMA, FP32 FMA, mma.sync m16n8k16 f16 -> f32 and half -> float conversion
// rates on the current device, each a 1-13 ms kernel timed with CUDA events.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe probe_throughput.cu
#include <cstdio>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)
template<typename T> __global__ void fma_kernel(T* out, int iters, T a, T b){
  T x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<16;j++){ x0=x0*a+b; x1=x1*a+b; x2=x2*a+b; x3=x3*a+b; x4=x4*a+b; x5=x5*a+b; x6=x6*a+b; x7=x7*a+b; }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void mma_kernel(float* out, int iters){
  unsigned a0=0x3c003c00u, a1=a0, a2=a0, a3=a0, b0=0x3c003c00u, b1=b0;
  float c[4][4]={};
  for(int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<4;j++){
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[j][0]),"+f"(c[j][1]),"+f"(c[j][2]),"+f"(c[j][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
    }
  }
  float s=0; for(int j=0;j<4;j++) s+=c[j][0]+c[j][1]+c[j][2]+c[j][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void cvt_kernel(float* out, const __half2* in, int iters){
  __half2 h = in[threadIdx.x & 31];
  float acc0=0, acc1=0, acc2=0, acc3=0;
  for(int i=0;i<iters;i++){
#pragma unroll
    for(int j=0;j<16;j++){ float2 f=__half22float2(h); acc0+=f.x; acc1+=f.y; h = __hadd2(h, __float2half2_rn(1e-8f)); float2 g=__half22float2(h); acc2+=g.x; acc3+=g.y; }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=acc0+acc1+acc2+acc3;
}
int main(){
  int nsm; CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
  int clk; CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
  printf("SMs %d clock(kHz attr) %d\n", nsm, clk);
  int blocks = nsm*8, threads=256; size_t n=(size_t)blocks*threads;
  double* dd; float* df; __half2* hin;
  CK(cudaMalloc(&dd, n*sizeof(double))); CK(cudaMalloc(&df, n*sizeof(float))); CK(cudaMalloc(&hin, 64*sizeof(__half2)));
  CK(cudaMemset(hin, 0, 64*sizeof(__half2)));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int rep=0;rep<2;rep++){
    int it64=200;
    fma_kernel<double><<<blocks,threads>>>(dd,it64,1.0000001,1e-9); CK(cudaGetLastError());
    cudaEventRecord(e0); fma_kernel<double><<<blocks,threads>>>(dd,it64,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double fl=2.0*n*it64*16*8; printf("FP64 FMA: %.3f ms, %.2f TFLOP/s\n", ms, fl/ms/1e9);
    int it32=4000;
    fma_kernel<float><<<blocks,threads>>>(df,it32,1.0000001f,1e-9f);
    cudaEventRecord(e0); fma_kernel<float><<<blocks,threads>>>(df,it32,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); fl=2.0*n*it32*16*8; printf("FP32 FMA: %.3f ms, %.2f TFLOP/s\n", ms, fl/ms/1e9);
    int itm=4000;
    mma_kernel<<<blocks,threads>>>(df,itm);
    cudaEventRecord(e0); mma_kernel<<<blocks,threads>>>(df,itm); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); fl=(double)blocks*(threads/32)*itm*4*2.0*16*8*16; printf("mma.sync m16n8k16 f16: %.3f ms, %.2f TFLOP/s, %.3f G mma/s\n", ms, fl/ms/1e9, fl/4096/ms/1e6);
    int itc=2000;
    cvt_kernel<<<blocks,threads>>>(df,hin,itc);
    cudaEventRecord(e0); cvt_kernel<<<blocks,threads>>>(df,hin,itc); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); double ncv=(double)n*itc*16*4; printf("half2->float2 cvt loop: %.3f ms, %.2f T cvt/s\n", ms, ncv/ms/1e9);
  }
  CK(cudaDeviceSynchronize());
  printf("OK\n");
  return 0;
}
