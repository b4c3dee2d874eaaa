/*
 * spx_probe.h - throughput probes behind the roofline denominators.
 *
 * The paper has no counterpart: these calls measure the B300's FP64 and
 * FP32 pipes, global atomics and the kernel launch rate, which the roofline
 * fractions reported by the benchmark are divided by.  Each call runs on its
 * own stream of the current device, allocates 1 MiB of device scratch, and
 * synchronises before returning.
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
  SPX_PROBE_LAUNCH = 5           /* empty <<<1,32>>> launches: launches/s   */
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
