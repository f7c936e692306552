/*
 * schedgpu.h -- C ABI of a memory-safe GPU co-scheduler for one B300
 * (sm_103a), following the life cycle of schedGPU (arXiv 1712.04495,
 * Sec. II and Sec. IV): initialise, pre-allocate (declare a device-memory
 * need and wait for the grant), run, post-free (release), shut down.
 *
 * Conventions for every call:
 *   - Return value: SG_OK (0) or one of the SG_* error codes below; nothing
 *     aborts the process. sg_strerror() names a code.
 *   - Pointers are plain host or device addresses as stated per argument;
 *     sizes are bytes unless named otherwise. Streams are cudaStream_t
 *     handles passed as void* (NULL = the legacy default stream).
 *   - The library never allocates device memory after sg_init(); the pool
 *     belongs to the caller and must outlive the context.
 *   - Calls on one context are safe from several host threads (the paper's
 *     "clients" are threads of one process here).
 */
#ifndef SCHEDGPU_H
#define SCHEDGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ codes */
/* Error codes mirror the CUDA codes the paper's API returns (Sec. IV):
 * cudaSuccess -> SG_OK, cudaErrorNotReady -> SG_NOT_READY (non-blocking
 * pre-allocation that cannot be served), cudaErrorUnknown -> SG_ERR_UNKNOWN. */
#define SG_OK             0
#define SG_NOT_READY      1  /* request queued, not granted yet                  */
#define SG_ERR_TIMEOUT    2  /* blocking wait expired; the ticket is withdrawn   */
#define SG_ERR_TOO_LARGE  3  /* need exceeds the whole pool; never queued        */
#define SG_ERR_INVALID    4  /* bad argument, unknown ticket, double release     */
#define SG_ERR_CUDA       5  /* a CUDA runtime call or launch failed             */
#define SG_ERR_UNKNOWN    6  /* internal error                                   */
#define SG_ERR_CAPACITY   7  /* ticket table of the context is full              */
#define SG_ERR_DEVICE     8  /* the device engine raised an error flag           */

/* Notification policies of Sec. V. A smaller priority value is a higher
 * priority (the priority argument of the paper's initialisation call). */
#define SG_POLICY_FIFO            0  /* Policy 1: serve the head while it fits      */
#define SG_POLICY_FIRST_FIT       1  /* Policy 2, MMU: serve every waiter that fits */
#define SG_POLICY_PRIO_FIFO       2  /* Policy 3: FIFO over (priority, arrival)     */
#define SG_POLICY_PRIO_FIRST_FIT  3  /* Policy 4: first fit in the top class        */

/* sg_config.flags */
#define SG_FLAG_FIFO_BYPASS  1u  /* FIFO: an arrival that fits is served even if
                                    others wait (the literal Sec. IV check)      */

/* Ticket / job states (sg_record.status). */
#define SG_ST_PENDING    0
#define SG_ST_QUEUED     1
#define SG_ST_RUNNING    2   /* granted, memory held */
#define SG_ST_DONE       3   /* released             */
#define SG_ST_TIMEOUT    4
#define SG_ST_TOO_LARGE  5

/* Job kinds run by sg_launch / sg_run_trace. */
#define SG_KIND_TRIAD 0      /* FP32 STREAM triad a = b + 3 c              */
#define SG_KIND_SPMV  1      /* FP32 CSR SpMV y = A x                      */
#define SG_KIND_GEMM  2      /* BF16 GEMM C = A B^T, FP32 accumulation     */

/* sg_run_trace.mode */
#define SG_RUN_SATURATED  1u  /* every job arrives at t = 0                        */
#define SG_RUN_TIMED      2u  /* jobs arrive at their arrival_ns (host clock)      */
#define SG_RUN_EXCLUSIVE  4u  /* each job declares the whole pool (one at a time)  */
#define SG_RUN_HOST_IO    8u  /* jobs / log / keep are HOST buffers, copied inside */
#define SG_RUN_KEEP      16u  /* write a digest of each job's output before release */

/* One job of a trace: 64 bytes, little-endian, no padding. The layout of a
 * job's data inside its grant and the generator of its inputs are fixed by
 * the kind (see sg_gen_* below). */
typedef struct sg_job {
    uint64_t arrival_ns;   /* arrival time on the trace clock              */
    uint64_t need;         /* declared bytes (rounded up to the granule)   */
    uint64_t duration_ns;  /* declared duration: the replay clock; the runner treats >= 1 ms as a long job */
    uint64_t timeout_ns;   /* UINT64_MAX = wait forever; 0 = non-blocking  */
    uint64_t key;          /* SplitMix64 key of the job's data             */
    uint64_t p0;           /* triad n | spmv rows | gemm M                 */
    uint64_t p1;           /* spmv nnz capacity | gemm N                   */
    uint32_t p2;           /* spmv Poisson table index | gemm K            */
    uint16_t kind;         /* SG_KIND_*                                    */
    int16_t  prio;         /* smaller = higher priority                    */
} sg_job;

/* Per-ticket log entry: 48 bytes. Times are the trace clock (replay) or
 * %globaltimer ns (real runs). */
typedef struct sg_record {
    int32_t  status;       /* SG_ST_*                                      */
    int32_t  slot;         /* real runs: stream slot the job ran on, else -1 */
    int64_t  grant_seq;    /* order of grants, -1 if never granted         */
    uint64_t grant_t;
    uint64_t offset;       /* byte offset of the grant in the pool         */
    uint64_t done_t;       /* release time (or timeout time)               */
    uint64_t arrival_t;
} sg_record;

typedef struct sg_config {
    uint32_t policy;       /* SG_POLICY_*                                  */
    uint32_t flags;        /* SG_FLAG_*                                    */
    uint32_t max_tickets;  /* tickets in use at once (0 = 1 << 17, <= 1 << 24) */
    uint32_t n_streams;    /* stream slots for sg_run_trace's non-GEMM jobs (0 = 4) */
    uint64_t granule;      /* allocation granule, power of two >= 256 (0 = 256) */
    uint32_t n_gemm_streams; /* high-priority slots for GEMM jobs (0 = 4)  */
    uint16_t run_flags;    /* SG_RUNF_*: when sg_run_trace starts admitted jobs (0 = default) */
    uint16_t phase_jobs;   /* starts of one kind per SpMV / GEMM phase while the other kind waits (0 = 64) */
} sg_config;

/* sg_config.run_flags. By default sg_run_trace never runs an SpMV job and a
 * GEMM job at the same time: it alternates phases of the two kinds, and
 * triads run beside either. A phase ends when its kind has no admitted job
 * left to start, or after phase_jobs starts while the other kind has
 * admitted jobs waiting; the next phase starts once the last job of the
 * previous one has finished. Admission is decided as before (the policy
 * pass and the placement); the rule only decides when an admitted job
 * starts, which in a real run moves its release and so later grants. On B300 an SpMV's random gathers and a GEMM's operand stream
 * both load L2; on the mixed trace, running the two kinds in turn finishes
 * sooner and with a shorter tail turnaround under load than overlapping
 * them. Jobs declared to run 1 ms or longer (sg_job.duration_ns) also run
 * one at a time, with shorter jobs beside them: each fills the GPU on its
 * own, and two together finish later than one after the other.
 * SG_RUNF_OVERLAP turns both rules off and starts every admitted job as soon
 * as a slot frees. */
#define SG_RUNF_OVERLAP  1u

typedef struct sg_grant {
    uint64_t offset;       /* byte offset in the pool                      */
    void*    ptr;          /* device pointer = pool + offset; valid until release */
    uint64_t grant_time_ns;
} sg_grant;

typedef struct sg_ctx sg_ctx;
typedef uint32_t sg_ticket;

typedef struct sg_run_stats {
    uint64_t elapsed_ns;       /* CUDA-event time from first declare to last release */
    uint64_t makespan_ns;      /* last release - first arrival (device clock)  */
    uint64_t wait_p50_ns, wait_p99_ns;             /* grant - arrival, nearest rank */
    uint64_t turnaround_p50_ns, turnaround_p99_ns; /* release - arrival           */
    uint64_t peak_used;        /* peak granted bytes                           */
    uint64_t frag_waits;       /* passes that ended blocked by fragmentation: the
                                  waiter the policy serves next fits the free
                                  byte count but no free extent holds it (a
                                  diagnostic of this library; the paper counts
                                  bytes only) */
    uint64_t launches;         /* kernels this call launched                   */
    uint64_t passes;           /* notification passes run by the engine        */
    uint32_t jobs_done, jobs_failed;
} sg_run_stats;

/* ------------------------------------------------------- life cycle */
/* Initialisation (Sec. IV, the paper's schedGPUInit). Creates a context
 * whose engine state -- budget, used bytes, per-ticket grants, the wait
 * queue and the free-extent list: the shared data of Sec. III-B -- lives in
 * device memory allocated here, once. dev_pool: device pointer, 256-byte
 * aligned, pool_bytes long (at most 2^47 granules), owned by the caller,
 * who keeps it allocated until sg_shutdown. When dev_pool is aligned to the
 * device's texture alignment (512 bytes), texture windows are made over the
 * pool for the SpMV's x gathers (1-D textures, no device memory); they go
 * with the context. cfg may be NULL for defaults. *out receives the
 * context. Errors:
 * SG_ERR_INVALID (null/misaligned/oversized pool, bad config), SG_ERR_CUDA. */
int sg_init(sg_ctx** out, void* dev_pool, uint64_t pool_bytes, const sg_config* cfg);

/* Shutdown (Sec. IV): waits for the context's streams, releases every
 * ticket still holding memory (notifying waiters), and frees the context
 * (never the pool). */
int sg_shutdown(sg_ctx* ctx);

/* Forget every ticket and return the pool to one free extent. Only valid
 * when no job of the context is in flight. Synchronous. */
int sg_reset(sg_ctx* ctx);

/* Pre-allocation, first half (Sec. IV, preCudaMalloc): declare a need of
 * `need` bytes with `priority` (-32768..32767, smaller = served first
 * under the priority policies); the device engine queues the request and
 * runs the admission pass. A grant never notifies other waiters.
 * Returns SG_OK with *out set (the request may already be granted; check
 * with sg_try), SG_ERR_TOO_LARGE at once if the need exceeds the pool,
 * SG_ERR_CAPACITY if max_tickets tickets are in use, SG_ERR_INVALID for a
 * priority out of range. A ticket is in use until its full release has run
 * on the device (sg_release with bytes = 0, or the job launched with
 * sg_launch finishing) or its request timed out; after that a later
 * sg_declare may hand out the same ticket number. */
int sg_declare(sg_ctx* ctx, uint64_t need, int32_t priority, sg_ticket* out);

/* Non-blocking check (Sec. IV: a non-blocking pre-allocation returns
 * cudaErrorNotReady): SG_OK and *out filled if granted, SG_NOT_READY if
 * still queued, SG_ERR_TIMEOUT if withdrawn, SG_ERR_INVALID otherwise. */
int sg_try(sg_ctx* ctx, sg_ticket t, sg_grant* out);

/* Blocking pre-allocation bounded by timeout_ns (Sec. IV and its footnote:
 * a timeout avoids deadlock). On expiry the ticket is withdrawn from the
 * device queue (which re-runs the notification pass) and SG_ERR_TIMEOUT is
 * returned -- unless the grant won the race, then SG_OK. */
int sg_wait(sg_ctx* ctx, sg_ticket t, uint64_t timeout_ns, sg_grant* out);

/* Post-free (Sec. IV, postCudaFree): enqueue on `stream`, after the work
 * that uses the memory, the release of `bytes` declared bytes of ticket t.
 * 0, or at least the bytes t still holds, frees everything (the paper's
 * bytes == 0 form); a smaller amount shrinks the grant from its end: t
 * keeps its first (held - bytes) bytes, rounded up to the granule, at the
 * same offset. Freeing notifies the waiters through the policy pass on the
 * device. SG_ERR_INVALID if t holds no memory (the paper's check that the
 * bytes were pre-allocated), including any release after a full one. */
int sg_release(sg_ctx* ctx, sg_ticket t, uint64_t bytes, void* stream);

/* Withdraw a request that is still waiting (what an expired blocking
 * pre-allocation does, Sec. IV): the engine removes it from the queue and
 * re-runs the notification pass. Returns SG_ERR_TIMEOUT if it was
 * withdrawn, SG_OK (with *out, may be NULL) if it had already been granted,
 * SG_ERR_INVALID for an unknown ticket. Synchronous. */
int sg_cancel(sg_ctx* ctx, sg_ticket t, sg_grant* out);

/* The grant notifications of Sec. IV (the paper's signal to a waiting
 * client): copies up to `max` tickets granted since *cursor, in grant order,
 * into out[], advances *cursor and sets *n_out. Start with *cursor = 0
 * after sg_init or sg_reset. Non-blocking, host only. SG_ERR_CAPACITY if
 * more than max_tickets grants were not read in time (the ring wrapped),
 * SG_ERR_DEVICE after a device engine error. */
int sg_poll_grants(sg_ctx* ctx, uint32_t* cursor, sg_ticket* out, uint32_t max, uint32_t* n_out);

/* Run job `job` in the memory granted to ticket t, on `stream`: its input
 * generator, then its kernel, whose last block releases the ticket
 * (wake-on-release without a host round trip). This is the application's
 * part of the life cycle between pre-allocation and post-free (Sec. VI,
 * "Concurrent Execution of Individual Applications": pre-allocation before
 * the allocations, post-free after the release of memory). tables_dev: device array of
 * 64-entry uint64 Poisson tables (SpMV jobs), may be NULL otherwise. */
int sg_launch(sg_ctx* ctx, sg_ticket t, const sg_job* job, const uint64_t* tables_dev,
              void* stream);

/* Run a whole trace, the many co-scheduled instances of the paper's
 * evaluation (Sec. VI, "Workloads Comprising Multiple Applications"): declare
 * every job (at t=0 or at its arrival time), launch each as it is granted on
 * a free stream slot, under the start rules
 * of sg_config.run_flags (SpMV and GEMM in turn, long jobs one at a time),
 * until every job is released. Ticket i is job i. jobs/log: device buffers (host buffers with
 * SG_RUN_HOST_IO, copied in and out inside the call). log receives one
 * sg_record per job (device clock). keep (SG_RUN_KEEP): n uint64 output
 * digests (see sg_digest), else NULL. stats may be NULL. */
int sg_run_trace(sg_ctx* ctx, const sg_job* jobs, uint32_t n, const uint64_t* tables_dev,
                 uint32_t mode, sg_record* log, uint64_t* keep, sg_run_stats* stats);

/* Replay a trace on the device engine with the logical clock and declared
 * durations (no job runs): the admission log the oracle must reproduce bit
 * for bit. jobs_dev sorted by arrival_ns (ties by index); log_dev receives n
 * records; workspace_dev of sg_replay_workspace_bytes(n) bytes, owned by
 * the caller. One warp runs the whole event loop on `stream`. stats_dev:
 * 4 uint64 (peak_used, frag_waits, passes, error flags) or NULL.
 * SG_ERR_INVALID for a null pointer, a bad policy or granule, or a budget
 * above 2^47 granules. */
uint64_t sg_replay_workspace_bytes(uint32_t n);
int sg_replay(const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
              uint32_t policy, uint32_t flags, uint32_t exclusive, sg_record* log_dev,
              void* workspace_dev, uint64_t* stats_dev, void* stream);

/* sg_replay without any allocation. The paper has no counterpart; this
 * entry point is for callers that cannot call cudaMalloc: a process that has
 * already handed all of its device memory to the pool this library
 * schedules (any further allocation would fall outside the budget the
 * scheduler accounts for, and could fail or push a co-scheduled job out of
 * memory), and latency-critical host loops that must not enter the CUDA
 * allocator. The caller passes the jobs, the log and the stats as for
 * sg_replay; the workspace is a fixed array of 2048 KiB inside the
 * library's device image, which every GPU that loads the library holds
 * until the process exits. Up to SG_REPLAY_NOALLOC_MAX_JOBS jobs; larger
 * traces get SG_ERR_TOO_LARGE and nothing runs. The first call on each
 * device (and again after the device's context was reset) looks up the
 * array's device address; make that first call before any stream capture:
 * while `stream` is being captured the lookup is refused with
 * SG_ERR_INVALID. All calls share the array and it keeps the last call's
 * contents; the replay initialises what it reads, so no clearing is needed,
 * but calls that overlap on the GPU race on it: order them on one stream.
 * Like sg_replay, a call that finds a CUDA error already pending on the
 * thread reports SG_ERR_CUDA. */
#define SG_REPLAY_NOALLOC_MAX_JOBS 16384u
int sg_replay_noalloc(const sg_job* jobs_dev, uint32_t n, uint64_t budget, uint64_t granule,
                      uint32_t policy, uint32_t flags, uint32_t exclusive, sg_record* log_dev,
                      uint64_t* stats_dev, void* stream);

/* Flags raised by job kernels that gave up a bounded wait (the tcgen05
 * GEMM's mbarrier waits), OR-ed since the last call, then cleared.
 * Synchronous (device-wide). */
int sg_kernel_errors(uint32_t* flags_out);

/* ------------------------------------------- client processes (server) */
/* The paper's clients are separate application processes that share the
 * scheduler (Sec. III). Here one server process owns the pool and the
 * device engine, and clients reach it over a UNIX socket (SOCK_SEQPACKET).
 * The pool is mapped into each client through CUDA IPC, and clients run
 * their own kernels on their grants.
 *
 * A grant is pushed to its client as soon as the engine makes it; this
 * replaces the paper's signal. A request with a finite timeout is withdrawn
 * when the timeout expires.
 *
 * Dead-client check: the server takes each client's pid from the socket.
 * When a connection closes, the client's tickets stay held until that
 * process has exited, because its kernels may still run until then. After
 * that, waiting requests are withdrawn and grants released, which notifies
 * the other waiters. A process that closes its connection but keeps running
 * keeps its grants until it exits. */
typedef struct sg_server sg_server;
typedef struct sg_server_counters {
    uint64_t clients_accepted, clients_reaped, declares, grants, timeouts, releases, protocol_errors;
    uint32_t clients_open, tickets_open;
} sg_server_counts;

/* Serve ctx's pool at socket_path (created, replacing a stale socket file;
 * at most 107 bytes) on a service thread. Call it from a thread whose
 * current device is ctx's. Clients can map the pool only if it is device
 * memory that CUDA IPC can share (a cudaMalloc allocation or part of one;
 * otherwise sg_client_pool fails and grants carry ptr = NULL). ctx stays
 * usable in-process. SG_ERR_INVALID if the socket cannot be bound. */
int sg_server_start(sg_ctx* ctx, const char* socket_path, sg_server** out);
int sg_server_counters(sg_server* s, sg_server_counts* out);
/* Stop serving and free the server (not ctx; tickets of clients still
 * connected stay with ctx until sg_reset / sg_shutdown). */
int sg_server_stop(sg_server* s);

typedef struct sg_client sg_client;
/* Connect to a server. SG_ERR_UNKNOWN if it cannot be reached or stops
 * answering (30 s), on this and every later client call. */
int sg_client_connect(const char* socket_path, sg_client** out);
int sg_client_info(sg_client* c, uint64_t* pool_bytes, uint64_t* granule);
/* This process's device pointer to the pool (CUDA IPC mapping on the
 * current device, opened on the first call). Grants returned after this
 * call carry ptr = pool + offset. */
int sg_client_pool(sg_client* c, void** dev_ptr);
/* Pre-allocation request (sg_declare for a client process): the server's
 * engine queues it; it is withdrawn after timeout_ns if still waiting
 * (UINT64_MAX: never). */
int sg_client_declare(sg_client* c, uint64_t need, int32_t priority, uint64_t timeout_ns, sg_ticket* out);
/* SG_OK (granted, *out filled), SG_NOT_READY, SG_ERR_TIMEOUT (withdrawn),
 * SG_ERR_INVALID (not this client's ticket). */
int sg_client_try(sg_client* c, sg_ticket t, sg_grant* out);
/* sg_client_try that blocks up to max_block_ns for the grant; SG_NOT_READY
 * if it has not come by then. */
int sg_client_wait(sg_client* c, sg_ticket t, uint64_t max_block_ns, sg_grant* out);
/* Post-free (sg_release for a client): the caller's work on the grant must
 * be complete (synchronise its streams first). bytes = 0 releases all. */
int sg_client_release(sg_client* c, sg_ticket t, uint64_t bytes);
/* Close the connection (tickets still held stay with the server until this
 * process exits) and unmap the pool. */
int sg_client_close(sg_client* c);

/* ------------------------------------------- shared memory (no server) */
/* The distributed control of Sec. III-A: client processes share the
 * scheduler state (Sec. III-B) through one POSIX shared-memory segment and
 * each makes its own admission decisions on it (pre-allocation, post-free
 * and the policies of Sec. IV-V, the same semantics as the device engine's:
 * strict FIFO unless SG_FLAG_FIFO_BYPASS, granule-rounded needs, address-
 * ordered first-fit placement, so a grant is an offset in one pool).
 * Updates are serialised by a file lock that the kernel drops when its
 * holder dies; a waiting client sleeps on a futex in its ticket and the
 * process that grants it wakes it. Robustness (Sec. III-A): a backup copy is
 * written when a client closes; the structure is checked when a client opens
 * and after a holder died inside an update, and a corrupt state is rebuilt
 * from the ticket table, else restored from the backup, else initialised
 * afresh; a client that closes or has been blocked for 2 ms (then every
 * 20 ms) reclaims what processes that have exited still hold.
 * The admission runs on the host here (the device engine needs one owner
 * process: see sg_server_start). No call allocates device memory.
 * Tickets are (generation << 16 | slot): a ticket that ended reads as
 * SG_ERR_INVALID. Only the declaring process may release or withdraw it. */
typedef struct sg_shm sg_shm;
typedef struct sg_shm_counts {
    uint64_t budget, granule, used, peak_used, grants, passes, frag_waits;
    uint64_t reaped;       /* tickets reclaimed from processes that ended     */
    uint64_t rebuilt;      /* corrupt states rebuilt from the ticket table    */
    uint64_t restored;     /* ... restored from the backup                    */
    uint64_t reset;        /* ... initialised afresh                          */
    uint64_t abandoned;    /* locks taken over from a holder that died mid-update */
    uint64_t timeouts, backups, generation;
    uint32_t policy, max_tickets, waiting, running, free_extents, reserved;
} sg_shm_counts;
/* Integrity problems reported by sg_shm_check */
#define SG_SHM_BAD_HEADER   1u
#define SG_SHM_BAD_TICKETS  2u
#define SG_SHM_BAD_USED     4u
#define SG_SHM_BAD_EXTENTS  8u
#define SG_SHM_BAD_QUEUE   16u
#define SG_SHM_BAD_SLOTS   32u
#define SG_SHM_DIRTY       64u   /* a holder died inside an update */
/* Create (budget > 0, the segment does not exist) or attach to the segment
 * `name` ("/name", POSIX shm; its backup is "/name.bak"). budget = 0 attaches
 * only; with budget > 0 an existing segment must have the same budget,
 * policy and granule, else SG_ERR_INVALID. cfg (may be NULL): max_tickets
 * (tickets in use at once, 0 = 4096, <= 65536), granule, flags. SG_ERR_UNKNOWN
 * if the segment cannot be mapped or locked within 10 s. */
int sg_shm_open(const char* name, uint64_t budget, uint32_t policy, const sg_config* cfg, sg_shm** out);
/* Pre-allocation: SG_OK and *out (granted at once or queued; see sg_shm_try),
 * SG_ERR_TOO_LARGE (need > budget, not queued), SG_ERR_CAPACITY, SG_ERR_INVALID
 * (priority outside 16 bits). */
int sg_shm_declare(sg_shm* s, uint64_t need, int32_t priority, sg_ticket* out);
/* Non-blocking: SG_OK (*out filled; ptr = pool + offset once the pool is
 * mapped in this process, else NULL), SG_NOT_READY, SG_ERR_INVALID (ended). */
int sg_shm_try(sg_shm* s, sg_ticket t, sg_grant* out);
/* Block up to timeout_ns (UINT64_MAX = forever) for the grant. On expiry the
 * request is withdrawn (the pass re-runs) and SG_ERR_TIMEOUT is returned,
 * unless the grant won the race (SG_OK). */
int sg_shm_wait(sg_shm* s, sg_ticket t, uint64_t timeout_ns, sg_grant* out);
/* Post-free of `bytes` (0 or >= held: all, the ticket ends); a partial release
 * keeps the granule-rounded rest at the front. SG_ERR_INVALID if t is not a
 * running ticket of this process. The caller's work on the grant must be
 * complete. */
int sg_shm_release(sg_shm* s, sg_ticket t, uint64_t bytes);
/* Snapshot of a live ticket: status, grant order, offset, grant and arrival
 * times (CLOCK_MONOTONIC ns); slot = -1, done_t = 0. SG_ERR_INVALID if ended. */
int sg_shm_record(sg_shm* s, sg_ticket t, sg_record* out);
int sg_shm_stats(sg_shm* s, sg_shm_counts* out);
/* Bytes held by process pid (the itemised used memory of Sec. III-A). */
int sg_shm_used_by(sg_shm* s, int32_t pid, uint64_t* bytes);
/* Run the integrity check now and recover if needed; *problems (may be
 * NULL) gets the SG_SHM_* bits found (0 = consistent). */
int sg_shm_check(sg_shm* s, uint32_t* problems);
/* Publish the device pool (pool_bytes >= budget, device memory of this
 * process) through CUDA IPC; sg_shm_pool maps it in other processes. The
 * pool must outlive the clients' use of it; closing the publishing handle
 * withdraws it. SG_ERR_CUDA if the handle cannot be made. */
int sg_shm_set_pool(sg_shm* s, void* dev_pool, uint64_t pool_bytes);
/* This process's address of the published pool: SG_OK, SG_NOT_READY (none
 * published), SG_ERR_CUDA (cannot be mapped). The mapping lasts until close. */
int sg_shm_pool(sg_shm* s, void** ptr);
/* The client ends: its requests are withdrawn, its memory freed (waiters
 * notified), the holders checked and the state backed up; then unmapped.
 * The segment stays for the other clients. */
int sg_shm_close(sg_shm* s);
/* Remove the segment and its backup (clients that have it mapped keep it). */
int sg_shm_unlink(const char* name);

/* ------------------------------------------------------- batching */
/* One CUDA graph for a whole trace: a static co-schedule. plan (host, n
 * records) is the log of sg_replay on the same jobs and pool size: it
 * fixes each job's offset in the pool and the grant order. Every job
 * becomes a child graph (its generators, its kernel, and with keep_dev its
 * output digest into keep_dev[j]); a job depends on every job that used any
 * byte of its extent earlier in grant order, so jobs that share memory
 * never overlap in time and the others run concurrently. The graph owns no
 * memory: dev_pool (pool_bytes) and tables_dev must outlive it. Build once,
 * launch many times; keep_dev accumulates, so zero it before each launch.
 * Jobs the plan did not grant are left out. */
typedef struct sg_graph sg_graph;
int sg_graph_build(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                   const uint64_t* tables_dev, const sg_record* plan, uint64_t* keep_dev,
                   sg_graph** out);
/* Enqueue one run of the graph on stream (a cudaStream_t, NULL = legacy
 * default stream); asynchronous. SG_ERR_INVALID for a NULL or unbuilt graph,
 * SG_ERR_CUDA if the launch fails. */
int sg_graph_launch(sg_graph* g, void* stream);
/* Shape of the built graph: jobs in it, kernel nodes, dependency edges
 * between jobs. Any output pointer may be NULL. SG_ERR_INVALID if g is NULL. */
int sg_graph_info(const sg_graph* g, uint64_t* jobs, uint64_t* kernels, uint64_t* edges);
/* Free the graph and its executable instance; g is invalid afterwards. The
 * caller makes sure no launch of it is still running. SG_ERR_INVALID if NULL. */
int sg_graph_destroy(sg_graph* g);

/* The same plan run by one persistent grouped kernel: every job is a
 * short program of phases (generators, kernel, optional digest), each
 * phase a set of block-sized chunks; all blocks of one cooperative launch
 * pull chunks from a single device work queue. A job's first chunks are
 * queued when every earlier job that used any byte of its extent has
 * finished, and the block finishing a phase queues the next one, so the
 * batch runs with no host round trip and no launch per job. Arguments as
 * for sg_graph_build; the object allocates its own device state (queue,
 * dependency lists) once at build time, never at launch. GEMM jobs need
 * K % 8 == 0. sg_batch_launch zeroes keep_dev itself. sg_batch_status
 * (synchronous) reports finished jobs and error flags: SG_OK when every
 * planned job finished, SG_ERR_DEVICE otherwise. */
typedef struct sg_batch sg_batch;
int sg_batch_build(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                   const uint64_t* tables_dev, const sg_record* plan, uint64_t* keep_dev,
                   sg_batch** out);
/* Enqueue one run on stream (a cudaStream_t): the per-launch state reset
 * (dependency counters, seeded work queue, keep_dev zeroed; for an online
 * batch the engine re-armed) and then one cooperative launch of the
 * persistent kernel. Asynchronous; a batch object runs one launch at a time
 * (launches on one stream are ordered). SG_ERR_INVALID if b is NULL,
 * SG_ERR_CUDA if a copy or the launch fails. An empty batch returns SG_OK. */
int sg_batch_launch(sg_batch* b, void* stream);
/* After the launch has finished (synchronises through blocking copies): the
 * jobs that completed and the batch's error flags (SG_DEVERR_* bits, 0 =
 * none); either pointer may be NULL.
 * SG_OK when every planned (or, online, every declared) job finished with no
 * flag set, SG_ERR_DEVICE otherwise, SG_ERR_CUDA if the read fails. */
int sg_batch_status(sg_batch* b, uint64_t* jobs_done, uint32_t* err_flags);

/* A batch that admits on the device instead of from a plan: the batch owns
 * an engine (policy SG_POLICY_*, the pool as budget, granule 256) that holds
 * every job declared at t = 0. The persistent kernel's first policy pass
 * grants what fits. The worker that finishes a job releases its memory under
 * the engine lock, and the jobs that the release's notification pass grants
 * are enqueued at once. Nothing is planned in advance and the host is not
 * involved. Jobs as for sg_batch_build (host array);
 * SG_ERR_TOO_LARGE if a job could never fit the pool. Run it with
 * sg_batch_launch; sg_batch_status, sg_batch_info and sg_batch_destroy apply
 * as for a planned batch. */
int sg_batch_build_online(void* dev_pool, uint64_t pool_bytes, const sg_job* jobs, uint32_t n,
                          const uint64_t* tables_dev, uint32_t policy, uint64_t* keep_dev, sg_batch** out);
/* The admission log of the last launch of an online batch (n records, host
 * memory): grant order, grant and completion times (%globaltimer), offsets.
 * SG_ERR_INVALID for a planned batch. Synchronous. */
int sg_batch_records(sg_batch* b, sg_record* out);
/* jobs planned, chunks in the batch, workers (four per SM) of the launch */
int sg_batch_info(const sg_batch* b, uint64_t* jobs, uint64_t* chunks, uint64_t* workers);
int sg_batch_destroy(sg_batch* b);

/* Error flag bits, as reported by sg_device_error, sg_state, the runners'
 * stats and sg_batch_status (0 = none). */
#define SG_DEVERR_WAIT      1u   /* a bounded wait (engine lock, peer) gave up    */
#define SG_DEVERR_STATE     2u   /* a ticket was in a state the operation forbids */
#define SG_DEVERR_ORDER     4u   /* trace arrivals not in non-decreasing order    */
#define SG_DEVERR_EVENTS    8u   /* replay event heap full                        */
#define SG_DEVERR_NNZ      16u   /* a SpMV job generated more non-zeros than declared */
#define SG_DEVERR_CAPACITY 32u   /* a device queue or list ran out of room        */
#define SG_DEVERR_ITEM     64u   /* batch: a malformed work item                  */
/* Engine error flags of the context (0 = none). */
uint32_t sg_device_error(sg_ctx* ctx);

/* Post-mortem view of the device engine's scalar state (the shared data of
 * Sec. III-B). Taken after ctx's control stream and stream slots have
 * finished their work; jobs launched by the caller on other streams may
 * still change it. */
typedef struct sg_state_summary {
    uint64_t budget, used, peak_used, max_free_extent, grants, passes, frag_waits;
    uint32_t policy, free_extents, waiting, done, error_flags, reserved;
} sg_state_summary;
/* Fill *out (caller-owned) with the summary above. Synchronises ctx's
 * control stream and slots first. SG_ERR_INVALID for NULL arguments,
 * SG_ERR_CUDA if a synchronisation or the read fails. */
int sg_state(sg_ctx* ctx, sg_state_summary* out);
/* A static, NUL-terminated description of an SG_* code (never NULL; an
 * unknown code gives "unrecognised code"). The caller does not free it. */
const char* sg_strerror(int code);

/* ------------------------------------------------------ job kernels */
/* FP32 STREAM triad a[i] = b[i] + s*c[i], product and sum rounded
 * separately (no fused multiply-add). Device pointers, n elements;
 * 128-bit access when all three are 16-byte aligned. */
int sg_triad(float* a, const float* b, const float* c, float s, uint64_t n, void* stream);

/* Triad inputs of a job with data key `key`: b = U(stream 1), c = U(stream 2)
 * where U is uniform[-1,1) from SplitMix64, two elements per output: element
 * 2m from bits 40..63 of output m, element 2m + 1 from bits 8..31
 * (tracegen's element generator). */
int sg_gen_triad(float* b, float* c, uint64_t n, uint64_t key, void* stream);

/* FP32 CSR SpMV y = A x. row_ptr: rows+1 entries, int32 (ptr64 = 0) or
 * int64 (ptr64 = 1); col int32, val fp32 (nnz each); x, y fp32 (rows).
 * Square matrix; device pointers. When x lies inside the pool of a live
 * context (as it does for SpMV jobs, whose arrays sit in their grant), x is
 * gathered through a texture window over that pool, otherwise with global
 * loads; y is the same either way. A launch into a stream that is capturing
 * a CUDA graph always uses loads, so that the graph holds no texture of a
 * context and stays valid after sg_shutdown. */
int sg_spmv(const void* row_ptr, int ptr64, const int32_t* col, const float* val,
            const float* x, float* y, uint64_t rows, void* stream);

/* How sg_spmv (and every SpMV job) gathers an x of `rows` floats at device
 * address x when its stream is not capturing a graph: SG_GATHER_TEXTURE
 * through a texture window of a live context's pool, SG_GATHER_LOAD with
 * global loads (x outside every pool, in a pool whose base is not
 * texture-aligned, or too long for one window). */
#define SG_GATHER_LOAD    0
#define SG_GATHER_TEXTURE 1
int sg_spmv_gather_path(const float* x, uint64_t rows);

/* Build the CSR matrix and x of an SpMV job in its declared layout at
 * `base` (row_ptr, col, val, x, y, scan workspace; each 256-byte aligned;
 * col / val sized for nnz_cap entries, row_ptr int64 when nnz_cap >= 2^31):
 * row lengths by inverse CDF on table_dev (64 uint64 thresholds), columns
 * uniform in [0, rows), values N(0,1), x uniform[-1,1). Columns and values
 * are written for all nnz_cap slots (those past the matrix's non-zeros are
 * never read). If the generated row lengths sum to more than nnz_cap,
 * row_ptr is clamped to nnz_cap and a flag is OR-ed into err_dev (uint32,
 * may be NULL). The scan workspace and y are scratch until the SpMV. */
int sg_gen_spmv(void* base, uint64_t rows, uint64_t nnz_cap, const uint64_t* table_dev,
                uint64_t key, uint32_t* err_dev, void* stream);

/* BF16 GEMM on tcgen05 tensor cores: C[M x N] (fp32, row-major) =
 * A[M x K] (bf16, row-major) * B, with B given transposed as Bt[N x K]
 * (bf16, row-major, K contiguous). Any M, N; K a positive multiple of 8
 * (rows of A and Bt must start on 16-byte boundaries), else
 * SG_ERR_INVALID; pointers 16-byte aligned. Ragged tiles are zero-filled
 * by TMA and masked on store. */
int sg_gemm_bf16(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N,
                 uint32_t K, void* stream);

/* GEMM output tiles. A tile code is (rows << 16) | columns: 128 x 64,
 * 128 x 128, 128 x 256 and 256 x 256. The plain widths 64, 128 and 256 are
 * accepted for the 128-row tiles. */
#define SG_GEMM_TILE(m, n) ((((uint32_t)(m)) << 16) | (uint32_t)(n))

/* sg_gemm_bf16 with an explicit output tile (0 = sg_gemm_tile's choice).
 * SG_ERR_INVALID for a code that is not one of the four tiles. */
int sg_gemm_bf16_tiled(const uint16_t* A, const uint16_t* Bt, float* C, uint32_t M, uint32_t N,
                       uint32_t K, uint32_t tile, void* stream);
/* The tile code sg_gemm_bf16 uses for an M x N output: the autotuner's
 * choice if it has tuned that shape, else 256 x 256 when every SM gets a
 * tile, else the widest 128-row tile that half of the SMs get (at most 1/8
 * of a tile wasted on the edges), else 128 x 64. Host only. */
uint32_t sg_gemm_tile(uint32_t M, uint32_t N);

/* Autotuner for the GEMM output tile. shapes: n_shapes (M, N, K) triples
 * (host). For each shape, generates inputs in `scratch` (device, needs
 * 2MK + 2NK + 4MN bytes rounded to 256 B per array; shapes that do not fit
 * are skipped with chosen = 0), times every tile that fits the shape (one
 * warm-up, median of three CUDA-event timings on `stream`) and records the
 * fastest tile code for (M, N) in a process-wide table used by every later
 * GEMM launch. chosen (tile codes) / best_ms (host, n_shapes each) may be
 * NULL. Synchronous. */
int sg_autotune_gemm(const uint32_t* shapes, uint32_t n_shapes, void* scratch, uint64_t scratch_bytes,
                     uint32_t* chosen, float* best_ms, void* stream);
/* Forget every tuned shape. */
int sg_autotune_clear(void);

/* GEMM inputs: A[i,k] = bf16(V(stream 1, i*K+k)), Bt[j,k] = bf16(V(stream 2, j*K+k)),
 * V the 16-bit uniform b * 2^-15 - 1 with b bits 16 (e mod 4) .. +15 of
 * SplitMix64 output e / 4 (four elements per output), rounded to nearest
 * even. */
int sg_gen_gemm(uint16_t* A, uint16_t* Bt, uint32_t M, uint32_t N, uint32_t K, uint64_t key,
                void* stream);

/* Measurement kernel, not a step of the method (the paper has no
 * counterpart): it times the random gathers x[col[i]] that bound the CSR
 * SpMV job kernel, on the SpMV's own columns. out_dev[c] = sum of
 * x[col[i]] over i in [1024 c, 1024 (c + 1)) for the ceil(n / 1024) chunks
 * c; col (int32, n entries, 16-byte aligned, every entry in [0, x_len)),
 * x (fp32, x_len entries) and out_dev are device arrays owned by the
 * caller. x is gathered the way sg_spmv gathers it (a texture window when x
 * lies in a live context's pool and the stream is not capturing, else
 * loads). SG_ERR_INVALID for a null or
 * misaligned col, a null x or out_dev. */
int sg_gather_sum(const int32_t* col, const float* x, uint64_t x_len, uint64_t n, float* out_dev,
                  void* stream);

/* Order-independent 64-bit digest of `words` 32-bit words at dev_ptr:
 * sum over i of mix64((i << 32) | word_i), modulo 2^64, added into
 * *out_dev (device uint64). Equal outputs give equal digests. */
int sg_digest(const void* dev_ptr, uint64_t words, uint64_t* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SCHEDGPU_H */
