/*
 * helm_trace.h -- kernel tracing of libhelm (no counterpart in the paper; it measures
 * the library itself).
 *
 * Every kernel launch of the library is counted.  When tracing is enabled, each launch
 * is also bracketed by two CUDA events recorded on the launch's own stream, so that
 * helm_trace_read can report the device time of every kernel by name.  Tracing adds
 * two event records per launch; counting alone costs nothing measurable.
 */
#ifndef HELM_TRACE_H
#define HELM_TRACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    char name[48];        /* kernel name */
    int64_t launches;     /* launches since the last reset */
    double total_ms;      /* summed device time of the traced launches (0 if tracing was off) */
    int64_t timed;        /* launches that were timed */
    double flops;         /* useful floating-point operations of the timed launches, for kernels
                             that report them (the tensor-core GEMM: 8 M N K per complex product
                             term, 0 for the others) */
} helm_trace_entry;

/* Enable (on != 0) or disable per-launch event timing.  Enabling creates a pool of CUDA
 * events up front (16384), so that timed launches create none.  Host only; not thread safe
 * with concurrent library calls. */
void helm_trace_enable(int on);
/* Time only the launches of the kernel with this name (NULL or "": every kernel).  Returns 0,
 * or -1 if no kernel has that name.  Counting is unaffected. */
int32_t helm_trace_select(const char *kernel_name);
/* Forget all counts and timings. */
void helm_trace_reset(void);
/* Synchronise the device, fold the recorded events into per-kernel totals and copy up
 * to max entries (kernels with at least one launch) into out.  Returns the number of
 * entries written, or -1 on a CUDA error. */
int32_t helm_trace_read(helm_trace_entry *out, int32_t max);
/* Total kernel launches since the last reset. */
int64_t helm_launch_count(void);

typedef struct {
    int32_t kernel;       /* kernel index (helm_trace_kernel_name) */
    int32_t stream;       /* 0, 1, ...: order in which the launch's stream first appeared */
    double start_ms;      /* device start / end of the launch, relative to the start of the */
    double end_ms;        /* first timed launch since the last reset or read */
} helm_trace_event;

/* Synchronise the device and copy up to max timed launches recorded since the last
 * reset or read, in launch order, into out (the records stay for helm_trace_read).
 * Returns the number written, or -1 on a CUDA error. */
int32_t helm_trace_timeline(helm_trace_event *out, int32_t max);
/* Name of kernel index id, or NULL if out of range. */
const char *helm_trace_kernel_name(int32_t id);

#ifdef __cplusplus
}
#endif
#endif /* HELM_TRACE_H */
