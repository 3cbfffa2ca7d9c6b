// Measurement program (not part of the library): throughput of FP64 FMA (DFMA),
// FP64 mma.sync (m8n8k4, m16n8k4, m16n8k16) and FP32 FMA on the current GPU, and
// the latency of a dependent DFMA chain.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/p fp64_units.cu && /tmp/p
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<int CH>
__global__ void dfma_k(double* out, int iters, double s) {
  double a[CH];
  #pragma unroll
  for (int i=0;i<CH;i++) a[i] = threadIdx.x*1e-3 + i;
  for (int it=0; it<iters; it++) {
    #pragma unroll
    for (int i=0;i<CH;i++) a[i] = fma(a[i], s, 1e-9);
  }
  double r=0;
  #pragma unroll
  for (int i=0;i<CH;i++) r+=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=r;
}
template<int CH>
__global__ void ffma_k(float* out, int iters, float s) {
  float a[CH];
  #pragma unroll
  for (int i=0;i<CH;i++) a[i] = threadIdx.x*1e-3f + i;
  for (int it=0; it<iters; it++) {
    #pragma unroll
    for (int i=0;i<CH;i++) a[i] = fmaf(a[i], s, 1e-9f);
  }
  float r=0;
  #pragma unroll
  for (int i=0;i<CH;i++) r+=a[i];
  out[blockIdx.x*blockDim.x+threadIdx.x]=r;
}
// m8n8k4 f64: A 1 reg, B 1 reg, C/D 2 regs per thread
__global__ void dmma884_k(double* out, int iters) {
  double a = threadIdx.x*1e-3, b = 1.0 + threadIdx.x*1e-4;
  double c[8][2];
  #pragma unroll
  for (int i=0;i<8;i++){c[i][0]=0;c[i][1]=0;}
  for (int it=0; it<iters; it++) {
    #pragma unroll
    for (int i=0;i<8;i++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
        : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double r=0;
  #pragma unroll
  for (int i=0;i<8;i++) r+=c[i][0]+c[i][1];
  out[blockIdx.x*blockDim.x+threadIdx.x]=r;
}
// m16n8k4 f64: A 2 regs, B 1 reg, C 4 regs
__global__ void dmma1684_k(double* out, int iters) {
  double a0 = threadIdx.x*1e-3, a1=a0*0.5, b = 1.0 + threadIdx.x*1e-4;
  double c[4][4];
  #pragma unroll
  for (int i=0;i<4;i++) for(int j=0;j<4;j++) c[i][j]=0;
  for (int it=0; it<iters; it++) {
    #pragma unroll
    for (int i=0;i<4;i++)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3]) : "d"(a0), "d"(a1), "d"(b));
  }
  double r=0;
  #pragma unroll
  for (int i=0;i<4;i++) r+=c[i][0]+c[i][1]+c[i][2]+c[i][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=r;
}
// m16n8k16 f64: A 8 regs, B 4 regs, C 4 regs
__global__ void dmma16816_k(double* out, int iters) {
  double a[8], b[4];
  #pragma unroll
  for (int i=0;i<8;i++) a[i]=threadIdx.x*1e-3+i;
  #pragma unroll
  for (int i=0;i<4;i++) b[i]=1.0+threadIdx.x*1e-4+i;
  double c[2][4];
  #pragma unroll
  for (int i=0;i<2;i++) for(int j=0;j<4;j++) c[i][j]=0;
  for (int it=0; it<iters; it++) {
    #pragma unroll
    for (int i=0;i<2;i++)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
        : "d"(a[0]),"d"(a[1]),"d"(a[2]),"d"(a[3]),"d"(a[4]),"d"(a[5]),"d"(a[6]),"d"(a[7]),
          "d"(b[0]),"d"(b[1]),"d"(b[2]),"d"(b[3]));
  }
  double r=0;
  #pragma unroll
  for (int i=0;i<2;i++) r+=c[i][0]+c[i][1]+c[i][2]+c[i][3];
  out[blockIdx.x*blockDim.x+threadIdx.x]=r;
}

int main() {
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  printf("%s SMs=%d cc=%d.%d smemOptin=%zu L2=%d\n", p.name, p.multiProcessorCount, p.major, p.minor, p.sharedMemPerBlockOptin, p.l2CacheSize);
  int sms=p.multiProcessorCount;
  size_t nthr = (size_t)sms*16*256;
  double* dout; float* fout;
  CK(cudaMalloc(&dout, nthr*sizeof(double))); CK(cudaMalloc(&fout, nthr*sizeof(float)));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for (int bps : {1, 2, 4, 8, 16}) {
    int blocks = sms*bps, iters=4000;
    dfma_k<8><<<blocks,256>>>(dout, 10, 0.999); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dfma_k<8><<<blocks,256>>>(dout, iters, 0.999); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl = 2.0*8*iters*(double)blocks*256;
    printf("DFMA  blocks/SM=%2d : %8.3f ms  %8.2f GFLOP/s  (%.3f FMA/clk/SM @2070MHz)\n", bps, ms, fl/ms*1e-6, fl/2/(ms*1e-3)/sms/2.07e9);
  }
  for (int bps : {1, 4, 8}) {
    int blocks = sms*bps, iters=4000;
    ffma_k<8><<<blocks,256>>>(fout, 10, 0.999f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); ffma_k<8><<<blocks,256>>>(fout, iters, 0.999f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl = 2.0*8*iters*(double)blocks*256;
    printf("FFMA  blocks/SM=%2d : %8.3f ms  %8.2f GFLOP/s\n", bps, ms, fl/ms*1e-6);
  }
  for (int bps : {1, 4, 8}) {
    int blocks = sms*bps, iters=2000;
    dmma884_k<<<blocks,256>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dmma884_k<<<blocks,256>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl = 2.0*8*8*4*8.0*iters*(double)blocks*(256/32);
    printf("DMMA m8n8k4   blocks/SM=%2d : %8.3f ms  %8.2f GFLOP/s\n", bps, ms, fl/ms*1e-6);
  }
  for (int bps : {1, 4, 8}) {
    int blocks = sms*bps, iters=2000;
    dmma1684_k<<<blocks,256>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dmma1684_k<<<blocks,256>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl = 2.0*16*8*4*4.0*iters*(double)blocks*(256/32);
    printf("DMMA m16n8k4  blocks/SM=%2d : %8.3f ms  %8.2f GFLOP/s\n", bps, ms, fl/ms*1e-6);
  }
  for (int bps : {1, 4, 8}) {
    int blocks = sms*bps, iters=1000;
    dmma16816_k<<<blocks,256>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dmma16816_k<<<blocks,256>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    double fl = 2.0*16*8*16*2.0*iters*(double)blocks*(256/32);
    printf("DMMA m16n8k16 blocks/SM=%2d : %8.3f ms  %8.2f GFLOP/s\n", bps, ms, fl/ms*1e-6);
  }
  // single-SM DFMA latency-bound chain: 1 block, 32 threads, 1 chain
  {
    cudaEventRecord(e0); dfma_k<1><<<1,32>>>(dout, 100000, 0.999); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("DFMA dependent chain latency: %.2f ns per fma\n", ms*1e6/100000);
  }
  return 0;
}
