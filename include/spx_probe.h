/*
 * spx_probe.h - throughput and latency probes behind the roofline
 * denominators and the tile-kernel design.
 *
 * The paper has no counterpart: these calls measure the B300's FP64 and
 * FP32 pipes, global atomics and the kernel launch rate, which the roofline
 * fractions reported by the benchmark are divided by, and the FP64 and
 * barrier latencies that bound the in-tile triangular solves.  Each call
 * runs on its own stream of the current device, allocates 1 MiB of device
 * scratch, and synchronises before returning.
 */
#ifndef SPX_PROBE_H_
#define SPX_PROBE_H_

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SPX_PROBE_DFMA = 0,            /* FP64 FMA, SIMT pipe: rate in FLOP/s     */
  SPX_PROBE_DMMA = 1,            /* FP64 mma.sync m8n8k4: rate in FLOP/s    */
  SPX_PROBE_FFMA = 2,            /* FP32 FMA: rate in FLOP/s                */
  SPX_PROBE_ATOMIC_SAME = 3,     /* atomicAdd on one address: ops/s         */
  SPX_PROBE_ATOMIC_DISTINCT = 4, /* atomicAdd on 64 Ki addresses: ops/s     */
  SPX_PROBE_LAUNCH = 5,          /* empty <<<1,32>>> launches: launches/s   */
  /* Latency probes (one block of 256 threads on one SM): *rate receives SM
   * clock cycles per step instead of a rate. */
  SPX_PROBE_LAT_DFMA = 6,        /* dependent FP64 FMA chain, one thread    */
  SPX_PROBE_LAT_DDIV = 7,        /* dependent FP64 division chain           */
  SPX_PROBE_LAT_DSQRT = 8,       /* dependent FP64 square-root chain        */
  SPX_PROBE_LAT_SYNC = 9,        /* __syncthreads() of 256 threads          */
  SPX_PROBE_WARP_DFMA = 10,      /* cycles per warp FP64 FMA instruction,   */
                                 /* 8 warps x 8 independent chains          */
  SPX_PROBE_WARP_DDIV = 11,      /* cycles per warp FP64 division, same     */
  SPX_PROBE_LAT_DRCP = 12,       /* dependent __drcp_rn + multiply chain    */
  SPX_PROBE_LAT_DRSQRT = 13,     /* dependent rsqrt chain                   */
  SPX_PROBE_NBODY = 14,          /* the n-body interaction arithmetic (3 sub,
                                    r^2, sqrt, division, 3 mul, add, 3 FMA)
                                    on register data, all SMs: interactions/s,
                                    the ALU ceiling of SPX_OP_NBODY_*        */
  SPX_PROBE_WIDEN_CHECK = 15     /* the integer FP32 -> FP64 widening of the
                                    tensor-core epilogues against the
                                    hardware conversion, over all 2^32 FP32
                                    bit patterns: *rate = number of
                                    mismatches (NaNs compare as NaN), 0 when
                                    exact; iters is ignored                  */
};

/* Run probe `which` with `iters` inner iterations (or launches).  Writes the
 * rate to *rate and the timed duration to *ms.  Returns 0, -1 (bad
 * argument), -7 (CUDA error) or -9 (no device). */
int spx_probe(int which, int iters, double* rate, double* ms);

/* Number of SMs of the current device, or a negative code. */
int spx_device_sm_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SPX_PROBE_H_ */
