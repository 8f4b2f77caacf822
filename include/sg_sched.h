/*
 * sg_sched.h -- the native core of continuous batching for CA-step requests
 * on many resident gaskets (the serving loop's per-iteration work, in C++).
 *
 * The kernels are the batch steps of sg.h (sg_batch_ca_steps: one launch
 * over a prefix-summed work list of every gasket's lambda block space, the
 * block-space map of Theorem 1, with the gasket-restricted CA step of
 * sg_ca_step per gasket).  The paper has no counterpart for serving; this
 * header adds the host side that runs between launches:
 *
 *   - a FIFO of requests per gasket, each asking for k CA steps;
 *   - one iteration (sg_sched_step): every resident gasket with a queued
 *     request advances by min(fuse, steps left in its head request), so a
 *     gasket never steps past a request and every result is the plain
 *     per-gasket step sequence in the order its requests were queued.  One
 *     batched launch serves each class of advances that share a halo size:
 *     1 step, 2..4, 5..8 and 9..16 (each gasket runs its own step count
 *     within its launch: sg_batch_ca_plan_host with steps);
 *   - the work lists of an iteration are written into page-locked host memory
 *     and reach the device in one asynchronous copy, so an iteration does not
 *     wait for the previous one: the host may prepare iteration i + 1 while
 *     the device runs iteration i.
 *
 * Memory: sg_sched_create allocates the scheduler's own work-list memory (two
 * slots of page-locked host memory and two of device memory, a few bytes per
 * gasket); the gaskets' state buffers belong to the caller, who hands them in
 * with sg_sched_set_buffers and keeps them alive while they are set.  All
 * calls on one scheduler come from one host thread, and its launches go to
 * one stream (or streams the caller orders): the scheduler is not locked.
 *
 * Errors: SG_EINVAL for invalid arguments (nothing changes), SG_ECUDA when a
 * CUDA call fails (message in sg_last_error_string()).  A batched launch that
 * the library refuses fails the head requests of the gaskets it was for:
 * nothing ran for them, their states stay, and they are reported in the
 * step's result; the rest of the iteration goes on.
 */
#ifndef SG_SCHED_H
#define SG_SCHED_H

#include "sg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_sched sg_sched;  /* opaque */

/*
 * sg_batch_ca_plan_host -- sg_batch_ca_plan without the copy: the work list
 * of `count` gaskets is written into host_image (at least
 * sg_batch_workspace_bytes(count) bytes, any host memory, e.g. page-locked
 * for an asynchronous copy) and *plan describes it as if it were already in
 * `workspace` (device memory of workspace_bytes bytes, 16-byte aligned).  The
 * caller copies the image to the workspace before launching the plan.
 *
 * steps (host array, or NULL) gives every gasket its own step count, 1 ..
 * SG_FUSE_MAX: a launch of the plan with sg_batch_ca_steps(plan, parity, k)
 * then advances gasket i by steps[i] (the halo is sized for k), and requires
 * k >= every steps[i]; the largest is recorded in plan->reserved[0].  Such a
 * plan cannot be captured into a graph, and sg_batch_ca_step (one step) takes
 * it only when every steps[i] is 1.  NULL: every gasket takes the launch's k.
 * Other arguments and errors as sg_batch_ca_plan.  Host-only.
 */
SG_API sg_status sg_batch_ca_plan_host(int count, const int *levels, const int *steps,
                                       uint8_t *const *buf_a, uint8_t *const *buf_b, int rho,
                                       void *host_image, uint64_t image_bytes, void *workspace,
                                       uint64_t workspace_bytes, sg_batch_plan *plan);

/*
 * sg_sched_create -- a scheduler for `count` gaskets (1 .. 65535) of the given
 * levels (host array; log2(rho) <= level <= 16), stepped with rho x rho tiles
 * (16, 32 or 64), advancing a gasket by at most `fuse` steps per iteration
 * (1 .. SG_FUSE_MAX).  opts (may be NULL) are the launch options of every
 * batched launch.  No gasket is resident until sg_sched_set_buffers.
 */
SG_API sg_status sg_sched_create(int count, const int *levels, int rho, int fuse,
                                 const sg_launch_opts *opts, sg_sched **out);

/* Release the scheduler's memory (after the stream has passed its last
 * iteration; the call synchronises on its own copies first).  NULL: SG_EINVAL. */
SG_API sg_status sg_sched_destroy(sg_sched *s);

/*
 * sg_sched_set_buffers -- gasket g's two state buffers (device pointers, n*n
 * bytes each, n = 2^level, 16-byte aligned, distinct); `cur` holds its
 * current state.  Both NULL: g is not resident, and its queued requests wait
 * (sg_sched_waiting lists it).  The scheduler swaps the two after each
 * iteration that advances g; sg_sched_gasket reports which one is current.
 */
SG_API sg_status sg_sched_set_buffers(sg_sched *s, int g, uint8_t *cur, uint8_t *nxt);

/*
 * sg_sched_submit -- queue n requests (host arrays): request[i] asks for
 * steps[i] >= 1 CA steps of gasket[i].  Requests of one gasket run in the
 * order they are queued.  All are checked before any is queued.
 */
SG_API sg_status sg_sched_submit(sg_sched *s, int n, const int32_t *gasket,
                                 const int64_t *request, const int32_t *steps);

/* Gaskets with queued requests that are not resident: up to max ids into
 * out[], *n = how many were written. */
SG_API sg_status sg_sched_waiting(const sg_sched *s, int32_t *out, int max, int *n);

/* What the scheduler knows of gasket g. */
typedef struct sg_sched_gasket_info {
    int32_t level;
    int32_t queued;        /* requests queued (the head one included) */
    int32_t head_left;     /* steps left in the head request (0 when none) */
    int32_t resident;      /* buffers set */
    uint64_t cur, nxt;     /* device pointers: current state, the other buffer */
    uint64_t last_use;     /* the last iteration (1, 2, ...) that advanced or tried g; 0 never */
    uint64_t steps_done;   /* steps applied to g by this scheduler */
} sg_sched_gasket_info;

SG_API sg_status sg_sched_gasket(const sg_sched *s, int g, sg_sched_gasket_info *info);

/*
 * sg_sched_drop -- remove every queued request of gasket g (for a gasket
 * that cannot be made resident): their ids into request[] and the steps of
 * each that had already run into steps_run[] (arrays of `max` entries; max
 * must be >= the gasket's queued count), *n = how many.
 */
SG_API sg_status sg_sched_drop(sg_sched *s, int g, int64_t *request, int32_t *steps_run, int max,
                               int *n);

/* The outcome of one iteration.  The caller provides the arrays (entries
 * for every gasket: `count` each is always enough). */
typedef struct sg_sched_result {
    int64_t *completed;           /* requests whose last step this iteration ran */
    int32_t *completed_gasket;
    int64_t *failed;              /* requests failed by a refused launch */
    int32_t *failed_gasket;
    int32_t *failed_steps_run;    /* steps of each that had run before */
    int32_t max_entries;          /* length of each array above */
    int32_t n_completed;          /* out */
    int32_t n_failed;             /* out */
    int32_t active;               /* out: gaskets this iteration tried to advance */
    int32_t launches;             /* out: batched launches issued */
    uint64_t cell_steps;          /* out: sum over advanced gaskets of 3^level * steps */
    uint64_t iteration;           /* out: this iteration's number (1, 2, ...); 0: nothing to do */
} sg_sched_result;

/*
 * sg_sched_step -- one iteration on `stream` (see above).  Returns as soon
 * as the copy and the launches are enqueued; the results are in the state
 * buffers once the stream reaches this point, so a completed request's state
 * can be read (or copied, on the same stream) right after the call.  With
 * no resident gasket holding a request nothing is enqueued and
 * res->iteration is 0.  max_entries below the number of gaskets that may
 * complete or fail (the count of gaskets always suffices): SG_EINVAL before
 * anything is enqueued.
 */
SG_API sg_status sg_sched_step(sg_sched *s, void *stream, sg_sched_result *res);

/*
 * sg_sched_inject_launch_failure -- host-side fault injection for tests of
 * failure containment: the next batched launch whose group holds gasket g
 * is not issued and is handled as a launch the library refused (SG_ECUDA):
 * the head requests of that group fail, nothing runs on the device.
 */
SG_API sg_status sg_sched_inject_launch_failure(sg_sched *s, int g);

#ifdef __cplusplus
}
#endif

#endif /* SG_SCHED_H */
