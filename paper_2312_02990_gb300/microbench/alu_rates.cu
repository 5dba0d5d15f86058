// alu_rates.cu -- throughput of FP32, FP64 and conversion instructions per SM clock.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/alu_rates \
//   paper_2312_02990_gb300/microbench/alu_rates.cu && /tmp/alu_rates
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__device__ unsigned long long g_cyc[4096];
__device__ float g_sinkf[1<<20];
__device__ double g_sinkd[1<<20];
__device__ long long g_sinkl[1<<20];

template<int OP> __global__ void k(float seed, int n) {
  float f[8]; double d[8]; long long l[8]; int ii[8]; float2 f2[8];
  for (int i=0;i<8;i++){ f[i]=seed+i*0.001f+threadIdx.x*1e-6f; d[i]=f[i]; l[i]=i+threadIdx.x; ii[i]=i*3+threadIdx.x;
                         f2[i]=make_float2(f[i], f[i]+0.5f); }
  const float2 c1 = make_float2(0.9999f, 0.9998f), c2 = make_float2(0.0001f, 0.0002f);
  __syncthreads();
  unsigned long long t0 = clock64();
  for (int it=0; it<n; it++) {
#pragma unroll
    for (int i=0;i<8;i++) {
      if (OP==0) f[i] = fmaf(f[i], 0.9999f, 0.0001f);
      if (OP==1) d[i] = fma(d[i], 0.9999, 0.0001);
      if (OP==2) { f[i] = __int2float_rn(ii[i]); ii[i] += 7; }            // I2F + IADD
      if (OP==3) { ii[i] ^= __float2int_rn(f[i]); f[i] += 1.5f; }         // F2I + FADD + LOP
      if (OP==4) { l[i] ^= __float2ll_rn(f[i]); f[i] += 1.5f; }           // F2I.S64
      if (OP==5) { d[i] = (double)f[i] + d[i]*0.0; f[i] += 1.0f; }       // F2F.F64.F32 (+dmul/dadd)
      if (OP==6) { f[i] = (float)d[i]; d[i] += 1.0; }                     // F2F.F32.F64 + DADD
      if (OP==7) { f[i] = rintf(f[i]*1.0001f); }                          // FMUL+FRND
      if (OP==8) { ii[i] = ii[i]*3 + 7; }                                 // IMAD
      if (OP==9) { l[i] += (long long)ii[i]; ii[i] += 1; }                // 64-bit add
      if (OP==10) { f[i] = f[i] + 12582912.0f; f[i] -= 12582911.0f; }    // 2 FADD (magic round)
      if (OP==11) { d[i] = d[i] + 1.0000001; }                            // DADD
      if (OP==12) { f2[i] = __ffma2_rn(f2[i], c1, c2); }                  // FFMA2 (2 lanes of work)
      if (OP==13) { f2[i] = __fadd2_rn(f2[i], c2); }                      // FADD2
      if (OP==14) { f2[i] = __fmul2_rn(f2[i], c1); }                      // FMUL2
    }
  }
  unsigned long long t1 = clock64();
  float sf=0; double sd=0; long long sl=0;
  for (int i=0;i<8;i++){ sf+=f[i]+ii[i]+f2[i].x+f2[i].y; sd+=d[i]; sl+=l[i]; }
  int gid = blockIdx.x*blockDim.x+threadIdx.x;
  if (sf==12345.678f) g_sinkf[gid&1023]=sf;
  if (sd==12345.678) g_sinkd[gid&1023]=sd;
  if (sl==1234567) g_sinkl[gid&1023]=sl;
  if (threadIdx.x==0) g_cyc[blockIdx.x] = t1-t0;
}

template<int OP> void run(const char* name, int nsm, int bps, int tpb, int opsPerIter) {
  k<OP><<<nsm*bps, tpb>>>(1.0f, 16); cudaDeviceSynchronize();
  cudaEvent_t a,b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a);
  k<OP><<<nsm*bps, tpb>>>(1.0f, ITERS);
  cudaEventRecord(b); cudaEventSynchronize(b);
  float ms; cudaEventElapsedTime(&ms,a,b);
  unsigned long long cyc[4096]; cudaMemcpyFromSymbol(cyc, g_cyc, sizeof(unsigned long long)*nsm*bps);
  double mc=0; for(int i=0;i<nsm*bps;i++) if (cyc[i]>mc) mc=cyc[i];
  double ops = (double)bps*tpb*ITERS*8*opsPerIter;  // per SM, thread-ops
  double per_clk = ops/mc;   // thread-ops per SM clock
  double totalops = (double)nsm*bps*tpb*ITERS*8*opsPerIter;
  printf("%-28s thread-ops/clk/SM=%8.2f  warp-instr/clk/SM=%6.3f  Gop/s=%10.1f  ms=%.3f  cyc=%.0f  MHz~%.0f\n",
         name, per_clk, per_clk/32, totalops/ms/1e6, ms, mc, mc/(ms*1e3));
  cudaError_t e = cudaGetLastError(); if (e) printf("err %s\n", cudaGetErrorString(e));
}
int main(){
  cudaDeviceProp p; cudaGetDeviceProperties(&p,0);
  printf("%s SMs=%d cc=%d.%d smemPerBlockOptin=%zu smemPerSM=%zu regsPerSM=%d L2=%d clock(kHz)=%d\n", p.name, p.multiProcessorCount, p.major, p.minor,
         p.sharedMemPerBlockOptin, p.sharedMemPerMultiprocessor, p.regsPerMultiprocessor, p.l2CacheSize, 0);
  int n=p.multiProcessorCount;
  run<0>("FFMA f32",n,4,256,1);
  run<1>("DFMA f64",n,4,256,1);
  run<11>("DADD f64",n,4,256,1);
  run<2>("I2F s32 (+IADD)",n,4,256,1);
  run<3>("F2I s32 (+FADD+LOP)",n,4,256,1);
  run<4>("F2I s64 (+FADD+LOP64)",n,4,256,1);
  run<5>("F2F f32->f64 (+DFMA)",n,4,256,1);
  run<6>("F2F f64->f32 (+DADD)",n,4,256,1);
  run<7>("FRND (+FMUL)",n,4,256,1);
  run<8>("IMAD i32",n,4,256,1);
  run<9>("IADD64 (+IADD)",n,4,256,1);
  run<10>("2xFADD magic",n,4,256,2);
  run<12>("FFMA2 (2 FMA per instr)",n,4,256,2);
  run<13>("FADD2 (2 adds per instr)",n,4,256,2);
  run<14>("FMUL2 (2 muls per instr)",n,4,256,2);
  return 0;
}
