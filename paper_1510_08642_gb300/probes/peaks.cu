// Throughput probe for the roofline denominators: FP64 DFMA / DADD, FP32 FFMA,
// INT32 IMAD / IADD, INT8 mma.sync (m16n8k32) and FP64 mma.sync (m8n8k4).
// Each kernel runs independent dependency chains in every thread of a grid of
// 1..8 blocks per SM; best of 5 timed launches. Prints one JSON line.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
template<int ILP>
__global__ void k_dfma(double* out, int iters, double a, double b){
  double x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x*1e-3+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=fma(x[i],a,b);
  }
  double s=0; for(int i=0;i<ILP;i++) s+=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_dadd(double* out, int iters, double a, double b){
  double x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x*1e-3+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=__dadd_rn(x[i],a);
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=__dadd_rn(x[i],b);
  }
  double s=0; for(int i=0;i<ILP;i++) s+=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_ffma(float* out, int iters, float a, float b){
  float x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x*1e-3f+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=fmaf(x[i],a,b);
  }
  float s=0; for(int i=0;i<ILP;i++) s+=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_imad(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=x[i]*a+b;
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_iadd(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) x[i]=(x[i]^a)+b;
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_mma8(int* out, int iters, int a0){
  int c[ILP][4];
  for(int i=0;i<ILP;i++){c[i][0]=c[i][1]=c[i][2]=c[i][3]=0;}
  int a1=a0+1,a2=a0+2,a3=a0+3,b0=a0^5,b1=a0^7;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[i][0]),"+r"(c[i][1]),"+r"(c[i][2]),"+r"(c[i][3]) : "r"(a0),"r"(a1),"r"(a2),"r"(a3),"r"(b0),"r"(b1));
  }
  int s=0; for(int i=0;i<ILP;i++) s+=c[i][0]+c[i][1]+c[i][2]+c[i][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int ILP>
__global__ void k_mmaf64(double* out, int iters, double a0){
  double c[ILP][2];
  for(int i=0;i<ILP;i++){c[i][0]=c[i][1]=0;}
  double b0=a0*0.5;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c[i][0]),"+d"(c[i][1]) : "d"(a0),"d"(b0));
  }
  double s=0; for(int i=0;i<ILP;i++) s+=c[i][0]+c[i][1];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  int sms=p.multiProcessorCount; printf("{\"gpu\":\"%s\",\"sms\":%d",p.name,sms);
  void* buf; size_t nmax=(size_t)sms*8*1024; CK(cudaMalloc(&buf,nmax*16));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  auto timeit=[&](auto launch, double ops, const char* name){
    for(int w=0;w<2;w++) launch();
    float best=1e30;
    for(int r=0;r<5;r++){ cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1); float ms; cudaEventElapsedTime(&ms,e0,e1); if(ms<best) best=ms; }
    cudaError_t err=cudaGetLastError(); if(err!=cudaSuccess){printf(",\"%s_err\":\"%s\"",name,cudaGetErrorString(err)); return;}
    printf(",\"%s\":%.4g",name, ops/(best*1e-3)); fflush(stdout);
  };
  for(int bpsm: {1,2,4,8}){
    int blocks=sms*bpsm, th=256, it=2000;
    char nm[64];
    snprintf(nm,64,"dfma_per_s_b%d",bpsm);
    timeit([&]{k_dfma<8><<<blocks,th>>>((double*)buf,it,1.0000001,1e-9);}, (double)blocks*th*it*8, nm);
    snprintf(nm,64,"dadd_per_s_b%d",bpsm);
    timeit([&]{k_dadd<8><<<blocks,th>>>((double*)buf,it,1e-9,-1e-9);}, (double)blocks*th*it*16, nm);
  }
  {int blocks=sms*4, th=256, it=20000;
  timeit([&]{k_ffma<8><<<blocks,th>>>((float*)buf,it,1.0000001f,1e-9f);}, (double)blocks*th*it*8, "ffma_per_s");
  timeit([&]{k_imad<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "imad_per_s");
  timeit([&]{k_iadd<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*16, "iaddxor_per_s");
  }
  for(int bpsm: {1,4}){
    int blocks=sms*bpsm, th=256, it=2000; char nm[64];
    snprintf(nm,64,"mma_s8_ops_per_s_b%d",bpsm);
    timeit([&]{k_mma8<4><<<blocks,th>>>((int*)buf,it,0x01020304);}, (double)blocks*(th/32)*it*4*(2.0*16*8*32), nm);
    snprintf(nm,64,"dmma_flops_per_s_b%d",bpsm);
    timeit([&]{k_mmaf64<4><<<blocks,th>>>((double*)buf,it/4,1.5);}, (double)blocks*(th/32)*(it/4)*4*(2.0*8*8*4), nm);
  }
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf(",\"clock_khz\":%d}\n",clk);
  return 0;
}
