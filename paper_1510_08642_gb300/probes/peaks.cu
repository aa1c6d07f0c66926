// Throughput probe for the roofline denominators: FP64 DFMA / DADD, FP32 FFMA,
// INT32 IMAD / IADD, 64-bit mad.wide, mad.hi, the three-instruction
// multiword multiply-add step, INT8 mma.sync (m16n8k32) and FP64 mma.sync
// (m8n8k4).
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
// 64-bit multiply-add of 32-bit operands: x64 += lo32(x64) * a (mad.wide)
template<int ILP, bool SIGNED>
__global__ void k_imadwide(unsigned long long* out, int iters, unsigned a){
  unsigned long long x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++){
      if(SIGNED) asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(x[i]) : "r"((unsigned)x[i]), "r"(a));
      else asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(x[i]) : "r"((unsigned)x[i]), "r"(a));
    }
  }
  unsigned long long s=0; for(int i=0;i<ILP;i++) s^=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// high word of a 32 x 32-bit product plus an addend (mad.hi)
template<int ILP>
__global__ void k_imadhi(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned x[ILP];
  for(int i=0;i<ILP;i++) x[i]=threadIdx.x+i;
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++) asm("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(a), "r"(b));
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=x[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// one partial product into a three-word running sum with carries
// (mad.lo.cc, madc.hi.cc, madc.lo): counted as one step of three instructions
template<int ILP>
__global__ void k_comba(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned c0[ILP], c1[ILP], c2[ILP];
  for(int i=0;i<ILP;i++){c0[i]=threadIdx.x+i; c1[i]=i; c2[i]=0;}
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++)
      asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\tmadc.lo.u32 %2, %2, 1, 0;"
          : "+r"(c0[i]), "+r"(c1[i]), "+r"(c2[i]) : "r"(a ^ c2[i]), "r"(b));
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=c0[i]^c1[i]^c2[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// the same step with the carry captured by addc instead of madc.lo
template<int ILP>
__global__ void k_comba_addc(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned c0[ILP], c1[ILP], c2[ILP];
  for(int i=0;i<ILP;i++){c0[i]=threadIdx.x+i; c1[i]=i; c2[i]=0;}
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++)
      asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
          : "+r"(c0[i]), "+r"(c1[i]), "+r"(c2[i]) : "r"(a ^ c2[i]), "r"(b));
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=c0[i]^c1[i]^c2[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// high half only into a two-word sum (mad.hi.cc, addc)
template<int ILP>
__global__ void k_hi_addc(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned c1[ILP], c2[ILP];
  for(int i=0;i<ILP;i++){c1[i]=threadIdx.x+i; c2[i]=0;}
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++)
      asm("mad.hi.cc.u32 %0, %2, %3, %0;\n\taddc.u32 %1, %1, 0;"
          : "+r"(c1[i]), "+r"(c2[i]) : "r"(a ^ c2[i]), "r"(b));
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=c1[i]^c2[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// two-word add with carry written as multiply-by-one (madc.lo x, y, 1, x) or as addc
template<int ILP, bool MADC>
__global__ void k_addcarry(unsigned* out, int iters, unsigned a, unsigned b){
  unsigned x0[ILP], x1[ILP];
  for(int i=0;i<ILP;i++){x0[i]=threadIdx.x+i; x1[i]=i;}
  for(int it=0; it<iters; it++){
    #pragma unroll
    for(int i=0;i<ILP;i++){
      if(MADC) asm("add.cc.u32 %0, %0, %2;\n\tmadc.lo.u32 %1, %3, 1, %1;" : "+r"(x0[i]), "+r"(x1[i]) : "r"(a), "r"(b ^ x0[i]));
      else asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(x0[i]), "+r"(x1[i]) : "r"(a), "r"(b ^ x0[i]));
    }
  }
  unsigned s=0; for(int i=0;i<ILP;i++) s^=x0[i]^x1[i];
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
  timeit([&]{k_imadwide<8,false><<<blocks,th>>>((unsigned long long*)buf,it,12345u);}, (double)blocks*th*it*8, "imad_wide_u32_per_s");
  timeit([&]{k_imadwide<8,true><<<blocks,th>>>((unsigned long long*)buf,it,12345u);}, (double)blocks*th*it*8, "imad_wide_s32_per_s");
  timeit([&]{k_imadhi<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "imad_hi_per_s");
  timeit([&]{k_comba<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "comba_step_per_s");
  timeit([&]{k_comba_addc<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "comba_step_addc_per_s");
  timeit([&]{k_hi_addc<8><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "hi_addc_step_per_s");
  timeit([&]{k_addcarry<8,true><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "add2_madc1_per_s");
  timeit([&]{k_addcarry<8,false><<<blocks,th>>>((unsigned*)buf,it,12345u,678u);}, (double)blocks*th*it*8, "add2_addc_per_s");
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
