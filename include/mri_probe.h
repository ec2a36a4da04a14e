/*
 * mri_probe.h -- measurement utility of libmri (not part of the method; the
 * paper has no counterpart).  The fast path is bound by the FP64 FMA pipe, so
 * the benchmark measures that pipe's issue rate on the device it runs on and
 * uses it as the roofline peak.
 */
#ifndef MRI_PROBE_H
#define MRI_PROBE_H
#ifdef __cplusplus
extern "C" {
#endif

/* Time independent FP64 FMA chains on every SM of the current device (best of 3
 * launches, CUDA events on `stream`) and return the FMA rate in *fma_per_s
 * (multiply by 2 for flop/s).  scratch: device array of scratch_doubles doubles,
 * at least 2048 per SM, overwritten; iters: FMAs per chain (4096 takes a few ms).
 * Returns 0, -1 for bad arguments or -3 for a CUDA error. */
int mri_probe_fp64_fma(double* scratch, long long scratch_doubles, int iters, double* fma_per_s, void* stream);

/* The same chains with only the first active_lanes (1..32) lanes of every warp
 * running them, warps_per_sm (1..32) warps on each SM: the rate of lane FMAs in
 * *lane_fma_per_s.  On a device whose FP64 unit spends the same time on a warp
 * instruction whatever its active lanes, this rate is proportional to
 * active_lanes; the benchmark records it, because that cost model is what bounds
 * the fast path's fraction of the FP64 peak (partial passes over n = Ns + 1
 * unknowns, triangular solves, warp-uniform scalar work).  scratch: at least
 * 32 warps_per_sm doubles per SM.  Returns 0, -1 or -3. */
int mri_probe_fp64_lanes(double* scratch, long long scratch_doubles, int iters, int active_lanes, int warps_per_sm,
                         double* lane_fma_per_s, void* stream);

/* One warp running one dependent FP64 FMA chain of iters FMAs: SM clock cycles
 * per FMA in *cycles (synchronises `stream`).  scratch: at least 40 doubles.
 * Returns 0, -1 or -3. */
int mri_probe_fp64_latency(double* scratch, long long scratch_doubles, int iters, double* cycles, void* stream);

/* The FP64 exponential the rate kernels use (a table-driven method after Tang,
 * 1989, see fastmath.cuh), applied elementwise y[i] = exp(x[i]) on the device,
 * so that its accuracy can be checked against libm.  Returns 0, -1 or -3. */
int mri_probe_exp(const double* x, double* y, long long n, void* stream);

/* exp(x) and exp(-x) from one argument reduction, as the rate kernels form the
 * species factors exp(-g/RT) and their inverses: y[i] = exp(x[i]), z[i] =
 * exp(-x[i]).  Returns 0, -1 or -3. */
int mri_probe_exp_pair(const double* x, double* y, double* z, long long n, void* stream);

/* The FP64 natural logarithm the rate kernels use (table-driven, after Tang,
 * 1990, see fastmath.cuh), y[i] = log(x[i]) on the device, for the same check.
 * Returns 0, -1 or -3. */
int mri_probe_log(const double* x, double* y, long long n, void* stream);

/* Test hook: record `device` as the device a loaded mechanism belongs to and return
 * the device it was recorded on before (-1 for a NULL mechanism).  Every call that
 * uses a mechanism checks that its device is the current one; with this hook a
 * single-GPU test can make that check fail (and put the right device back after).
 * Nothing else reads the recorded device. */
typedef struct mri_mech mri_mech;
int mri_probe_mech_device(mri_mech* mech, int device);

#ifdef __cplusplus
}
#endif
#endif
