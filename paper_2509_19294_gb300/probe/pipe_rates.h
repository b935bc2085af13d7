/*
 * pipe_rates.h -- libnbody_probe.so: measured per-SM issue rates behind the
 * force kernel's roofline.  A measurement library used by the benchmark, not
 * part of the force library (libnbody.so) or its ABI (include/nbody.h).
 */
#ifndef NBODY_PIPE_RATES_H
#define NBODY_PIPE_RATES_H

#ifdef __cplusplus
extern "C" {
#endif

#define NBODY_PROBE_EINVAL (-1) /* out is NULL or n_out < 4 */
#define NBODY_PROBE_ENOMEM (-2) /* the probe's device buffers could not be allocated */
#define NBODY_PROBE_ECUDA (-3)  /* a CUDA runtime call or a probe launch failed */

/*
 * Per-SM issue rates of the current GPU, measured with one CTA per SM (1024
 * threads; 256 for the pair arithmetic, as the force kernel's C5 shapes run)
 * and clock64() cycles (so they do not depend on the clock frequency).
 * out (host, n_out >= 4):
 *   out[0] FP32 lane-operations per clock per SM with paired (f32x2) FMA
 *   out[1] MUFU rsqrt results per clock per SM
 *   out[2] pairwise interactions per clock per SM of the F32C kernel's per-pair
 *          arithmetic alone, potential terms summed as in its tile loop
 *          (register-resident operands, no shared-memory loads)
 *   out[3] FP64 FMA per clock per SM
 * Allocates and frees a small device buffer and synchronises the device.
 * Returns 0 or a negative NBODY_PROBE_E* code.
 */
int nbody_measure_pipes(double *out, int n_out);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_PIPE_RATES_H */
