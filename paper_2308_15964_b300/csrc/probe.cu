// Throughput probes for the roofline denominators that the driver does not
// measure: FP64 FMA on the SIMT pipe (DFMA), FP64 mma.sync (DMMA), FP32 FMA,
// global atomics on one address and on distinct addresses, and the launch
// rate of an empty kernel.  Each probe times itself with CUDA events on its
// own stream and returns a rate.  Declared in include/spx_probe.h.
#include <cuda_runtime.h>
#include <stdint.h>

#include "spx_probe.h"
#include "tile_tc.cuh"

namespace {

constexpr int kChains = 8;

__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[threadIdx.x] = s;  // keeps the loop alive
}

__global__ void ffma_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) out[threadIdx.x] = s;
}

// FP64 tensor MMA m8n8k4: D(8x8) = A(8x4) B(4x8) + C, per warp.
__global__ void dmma_kernel(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-3;
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) { d[c][0] = 0.0; d[c][1] = 0.0; }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
          : "+d"(d[c][0]), "+d"(d[c][1])
          : "d"(a), "d"(b));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  if (s == 12345.678) out[threadIdx.x] = s;
}

__global__ void atomic_same_kernel(unsigned* ctr, int iters) {
  for (int i = 0; i < iters; ++i) atomicAdd(ctr, 1u);
}

__global__ void atomic_distinct_kernel(unsigned* ctr, int iters, int n) {
  const int idx = (blockIdx.x * blockDim.x + threadIdx.x) % n;
  for (int i = 0; i < iters; ++i) atomicAdd(ctr + idx, 1u);
}

__global__ void empty_kernel() {}

// Every FP32 bit pattern: the integer widening against (double)f.
__global__ void widen_check_kernel(unsigned long long* bad) {
  unsigned long long nbad = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       i < (1ull << 32); i += (unsigned long long)gridDim.x * blockDim.x) {
    const float f = __uint_as_float((uint32_t)i);
    const double w = spx::widen_f32(f), h = (double)f;
    const bool ok = (f != f) ? (w != w) : (__double_as_longlong(w) == __double_as_longlong(h));
    nbad += ok ? 0u : 1u;
  }
  if (nbad) atomicAdd(bad, nbad);
}

// The interaction arithmetic of the n-body ops on register data: 4
// independent targets per thread against a moving source.
__global__ void nbody_probe_kernel(double* out, int iters, double qv) {
  double xi[4], phi[4], ex[4], ey[4], ez[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    xi[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    phi[c] = ex[c] = ey[c] = ez[c] = 0.0;
  }
  double sx = 0.25, sy = 0.5, sz = -0.125;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double dx = xi[c] - sx, dy = xi[c] - sy, dz = xi[c] - sz;
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const double rinv = 1.0 / sqrt(r2);
      const double qr = qv * rinv;
      const double s3 = qr * rinv * rinv;
      phi[c] += qr;
      ex[c] = fma(s3, dx, ex[c]);
      ey[c] = fma(s3, dy, ey[c]);
      ez[c] = fma(s3, dz, ez[c]);
    }
    sx += 1e-6;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += phi[c] + ex[c] + ey[c] + ez[c];
  if (s == 12345.678) out[threadIdx.x] = s;
}

// Latency probes: one block, thread 0 times a dependent chain with clock64()
// and writes the SM cycles per step to out[0].
enum LatOp { kLatDfma, kLatDdiv, kLatDsqrt, kLatSync, kLatWarpDfma, kLatWarpDdiv, kLatDrcp,
             kLatDrsqrt };

__global__ void latency_kernel(double* out, int iters, int op, double a, double b) {
  double x = 1.0 + threadIdx.x * 1e-9, y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) y[c] = x + c;
  __syncthreads();
  const long long t0 = clock64();
  switch (op) {
    case kLatDfma:
      for (int i = 0; i < iters; ++i) x = fma(x, a, b);
      break;
    case kLatDdiv:
      for (int i = 0; i < iters; ++i) x = a / x;
      break;
    case kLatDsqrt:
      for (int i = 0; i < iters; ++i) x = sqrt(x) + b;
      break;
    case kLatSync:
      for (int i = 0; i < iters; ++i) __syncthreads();
      break;
    case kLatWarpDfma:  // all threads, kChains independent chains each
      for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = fma(y[c], a, b);
      break;
    case kLatWarpDdiv:  // all threads, kChains independent divisions each
      for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) y[c] = a / y[c];
      break;
    case kLatDrcp:  // correctly rounded reciprocal
      for (int i = 0; i < iters; ++i) x = __drcp_rn(x) * a;
      break;
    default:  // kLatDrsqrt
      for (int i = 0; i < iters; ++i) x = rsqrt(x) + b;
      break;
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = x;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += y[c];
  if (s == 12345.678) out[1] = s;
  if (threadIdx.x == 0) {
    const bool warps = op == kLatWarpDfma || op == kLatWarpDdiv;
    const double steps = warps ? (double)iters * kChains * (blockDim.x / 32) : iters;
    out[0] = (double)(t1 - t0) / steps;
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  return sms;
}

}  // namespace

extern "C" int spx_probe(int which, int iters, double* rate, double* ms) {
  if (!rate || !ms || iters <= 0) return -1;
  const int sms = sm_count();
  if (sms <= 0) return -9;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return -7;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void* buf = nullptr;
  cudaMalloc(&buf, 1 << 20);
  cudaMemsetAsync(buf, 0, 1 << 20, st);
  const int blocks = sms * 8, threads = 256;
  double work = 0.0;
  for (int rep = 0; rep < 2; ++rep) {  // first pass warms up
    cudaEventRecord(e0, st);
    switch (which) {
      case SPX_PROBE_DFMA:
        dfma_kernel<<<blocks, threads, 0, st>>>((double*)buf, iters, 0.999999, 1e-7);
        work = 2.0 * kChains * (double)iters * blocks * threads;
        break;
      case SPX_PROBE_DMMA:
        dmma_kernel<<<blocks, threads, 0, st>>>((double*)buf, iters);
        work = 2.0 * 8 * 8 * 4 * 4.0 * (double)iters * blocks * (threads / 32);
        break;
      case SPX_PROBE_FFMA:
        ffma_kernel<<<blocks, threads, 0, st>>>((float*)buf, iters, 0.999999f, 1e-7f);
        work = 2.0 * kChains * (double)iters * blocks * threads;
        break;
      case SPX_PROBE_ATOMIC_SAME:
        atomic_same_kernel<<<sms * 2, 256, 0, st>>>((unsigned*)buf, iters);
        work = (double)iters * sms * 2 * 256;
        break;
      case SPX_PROBE_ATOMIC_DISTINCT:
        atomic_distinct_kernel<<<sms * 2, 256, 0, st>>>((unsigned*)buf, iters, 65536);
        work = (double)iters * sms * 2 * 256;
        break;
      case SPX_PROBE_LAUNCH:
        for (int i = 0; i < iters; ++i) empty_kernel<<<1, 32, 0, st>>>();
        work = iters;
        break;
      case SPX_PROBE_WIDEN_CHECK:
        widen_check_kernel<<<blocks, threads, 0, st>>>((unsigned long long*)buf);
        work = 0.0;
        break;
      case SPX_PROBE_NBODY:
        nbody_probe_kernel<<<blocks, threads, 0, st>>>((double*)buf, iters, 0.75);
        work = 4.0 * (double)iters * blocks * threads;
        break;
      case SPX_PROBE_LAT_DFMA:
      case SPX_PROBE_LAT_DDIV:
      case SPX_PROBE_LAT_DSQRT:
      case SPX_PROBE_LAT_SYNC:
      case SPX_PROBE_WARP_DFMA:
      case SPX_PROBE_WARP_DDIV:
      case SPX_PROBE_LAT_DRCP:
      case SPX_PROBE_LAT_DRSQRT:
        latency_kernel<<<1, 256, 0, st>>>((double*)buf, iters, which - SPX_PROBE_LAT_DFMA,
                                          1.0000001, 1e-9);
        work = 0.0;
        break;
      default:
        work = -1.0;
    }
    cudaEventRecord(e1, st);
  }
  cudaError_t err = cudaStreamSynchronize(st);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  double cyc = 0.0;  // latency probes: cycles per step, written by the kernel
  unsigned long long bad_count = 0;  // widening check: mismatches
  if (err == cudaSuccess && which == SPX_PROBE_WIDEN_CHECK)
    err = cudaMemcpy(&bad_count, buf, sizeof(bad_count), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && which >= SPX_PROBE_LAT_DFMA && which <= SPX_PROBE_LAT_DRSQRT)
    err = cudaMemcpy(&cyc, buf, sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (work < 0) return -1;
  if (err != cudaSuccess) return -7;
  *ms = t;
  const bool lat = which >= SPX_PROBE_LAT_DFMA && which <= SPX_PROBE_LAT_DRSQRT;
  *rate = lat ? cyc : work / (t * 1e-3);
  if (which == SPX_PROBE_WIDEN_CHECK) *rate = (double)bad_count;
  return 0;
}

extern "C" int spx_device_sm_count(void) { return sm_count(); }
