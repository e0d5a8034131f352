// GB300 microbenchmarks used for the design and the roofline denominators:
// FP64 DFMA and FP32 FFMA throughput, MUFU lg2 throughput, the issue interval
// of one FP64 / FP32 instruction from a single active lane, and L2-resident
// and HBM read bandwidth.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/gb300_probe \
//       paper_2402_06835_gb300/probe/gb300_probe.cu && /tmp/gb300_probe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int CH> __global__ void dfma_tp(double* out, int iters, double a, double b){
  double x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-3+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fma(x[c],a,b);
  }
  double s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int CH> __global__ void ffma_tp(float* out, int iters, float a, float b){
  float x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=threadIdx.x*1e-3f+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fmaf(x[c],a,b);
  }
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int CH> __global__ void mufu_tp(float* out, int iters){
  float x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=1.5f+threadIdx.x*1e-3f+c;
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=__log2f(x[c])+2.0f;
  }
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
// single active lane, CH independent chains: clocks per FP64 instruction
template<int CH> __global__ void dfma_lane(double* out, long long* clk, int iters, double a, double b){
  if(threadIdx.x!=0) return;
  double x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=c;
  long long t0=clock64();
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fma(x[c],a,b);
  }
  long long t1=clock64();
  double s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[0]=s; clk[0]=t1-t0;
}
template<int CH> __global__ void ffma_lane(float* out, long long* clk, int iters, float a, float b){
  if(threadIdx.x!=0) return;
  float x[CH];
  #pragma unroll
  for(int c=0;c<CH;c++) x[c]=c;
  long long t0=clock64();
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int c=0;c<CH;c++) x[c]=fmaf(x[c],a,b);
  }
  long long t1=clock64();
  float s=0;
  #pragma unroll
  for(int c=0;c<CH;c++) s+=x[c];
  out[0]=s; clk[0]=t1-t0;
}
__global__ void l2read(const float4* __restrict__ buf, size_t n, int reps, float* out){
  float acc=0;
  for(int r=0;r<reps;r++)
    for(size_t i=blockIdx.x*(size_t)blockDim.x+threadIdx.x;i<n;i+=(size_t)gridDim.x*blockDim.x){
      float4 v=__ldcg(buf+i); acc+=v.x+v.y+v.z+v.w;
    }
  if(acc==12345.f) out[0]=acc;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("name %s SMs %d l2 %d MB smemPerBlockOptin %zu\n",p.name,p.multiProcessorCount,p.l2CacheSize>>20,p.sharedMemPerBlockOptin);
  int sms=p.multiProcessorCount;
  double* dout; float* fout; long long* clk;
  CK(cudaMalloc(&dout,sizeof(double)*sms*8*1024)); CK(cudaMalloc(&fout,sizeof(float)*sms*8*1024)); CK(cudaMalloc(&clk,64));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  // FP64 throughput
  for(int rep=0;rep<2;rep++){
    int iters=20000; int blocks=sms*4, th=256;
    cudaEventRecord(e0); dfma_tp<8><<<blocks,th>>>(dout,iters,0.999999,1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*iters*(double)blocks*th; printf("FP64 DFMA: %.3f TFLOP/s (%.2f ms)\n",fl/ms/1e9,ms);
  }
  for(int rep=0;rep<2;rep++){
    int iters=20000; int blocks=sms*8, th=256;
    cudaEventRecord(e0); ffma_tp<8><<<blocks,th>>>(fout,iters,0.999999f,1e-7f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl=2.0*8*iters*(double)blocks*th; printf("FP32 FFMA: %.3f TFLOP/s (%.2f ms)\n",fl/ms/1e9,ms);
  }
  for(int rep=0;rep<2;rep++){
    int iters=4000; int blocks=sms*8, th=256;
    cudaEventRecord(e0); mufu_tp<8><<<blocks,th>>>(fout,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double op=8.0*iters*(double)blocks*th; printf("MUFU lg2: %.3f Tops/s (%.2f ms) = %.2f /clk/SM @2.0GHz\n",op/ms/1e9,ms, op/ms/1e3/sms/2.0e9);
  }
  // single lane latencies / issue
  long long hc;
  int iters=10000;
  dfma_lane<1><<<1,32>>>(dout,clk,iters,0.999999,1e-7); CK(cudaDeviceSynchronize()); cudaMemcpy(&hc,clk,8,cudaMemcpyDeviceToHost); printf("FP64 1 lane dep chain: %.2f clk/instr\n",(double)hc/iters);
  dfma_lane<8><<<1,32>>>(dout,clk,iters,0.999999,1e-7); CK(cudaDeviceSynchronize()); cudaMemcpy(&hc,clk,8,cudaMemcpyDeviceToHost); printf("FP64 1 lane 8 chains: %.2f clk/instr\n",(double)hc/iters/8);
  ffma_lane<1><<<1,32>>>(fout,clk,iters,0.999999f,1e-7f); CK(cudaDeviceSynchronize()); cudaMemcpy(&hc,clk,8,cudaMemcpyDeviceToHost); printf("FP32 1 lane dep chain: %.2f clk/instr\n",(double)hc/iters);
  ffma_lane<8><<<1,32>>>(fout,clk,iters,0.999999f,1e-7f); CK(cudaDeviceSynchronize()); cudaMemcpy(&hc,clk,8,cudaMemcpyDeviceToHost); printf("FP32 1 lane 8 chains: %.2f clk/instr\n",(double)hc/iters/8);
  // one warp, full lanes, 8 chains (per-warp FP64 issue rate)
  for(int w=1; w<=8; w*=2){
    int it=20000;
    cudaEventRecord(e0); dfma_tp<8><<<1,32*w>>>(dout,it,0.999999,1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("FP64 1 block %d warps x8 chains: %.2f ns per warp-instr-per-warp, %.3f GFLOP/s\n",w,ms*1e6/(it*8.0), 2.0*8*it*32*w/ms/1e6);
  }
  // L2 read bandwidth, 64 MB buffer resident
  size_t n=(64ull<<20)/16; float4* buf; CK(cudaMalloc(&buf,n*16)); CK(cudaMemset(buf,0,n*16));
  for(int rep=0;rep<3;rep++){
    int reps=20;
    cudaEventRecord(e0); l2read<<<sms*4,512>>>(buf,n,reps,fout); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("L2-resident read 64MB x%d: %.1f GB/s\n",reps,(double)n*16*reps/ms/1e6);
  }
  size_t n2=(2048ull<<20)/16; float4* buf2; CK(cudaMalloc(&buf2,n2*16)); CK(cudaMemset(buf2,0,n2*16));
  for(int rep=0;rep<3;rep++){
    cudaEventRecord(e0); l2read<<<sms*4,512>>>(buf2,n2,1,fout); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1); printf("HBM read 2GB: %.1f GB/s\n",(double)n2*16/ms/1e6);
  }
  return 0;
}
