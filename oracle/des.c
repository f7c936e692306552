/*
 * Oracle (test infrastructure only; never linked into the product path):
 * a plain discrete-event simulator of the schedGPU admission and
 * notification semantics on a logical integer clock (ns).
 *
 * What it follows (arXiv 1712.04495):
 *   - shared state of Sec. III-B: total memory, total used, per-client
 *     used, and a queue of waiting clients (with priority when the policy
 *     needs one);
 *   - pre-allocation of Sec. IV: a request is served when the requested
 *     memory is available, otherwise the client waits (blocking, bounded by
 *     its timeout) or gets "not ready"; a grant does not notify others;
 *   - post-free of Sec. IV: freeing memory notifies the waiting clients
 *     through the policy in use;
 *   - the four notification policies of Sec. V (FIFO, MMU, Priority FIFO,
 *     Priority MMU) and their recursive definitions;
 *   - exclusive use of the GPU by pre-allocating all of it (Sec. VIII).
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes): one policy pass per event, events at equal time ordered
 * completion < arrival < timeout then by job id; an arrival joins the tail
 * and the policy pass runs (so FIFO is strict unless FLAG_FIFO_BYPASS asks
 * for the literal "serve if memory is available" check at arrival);
 * requests larger than the pool fail at once; a timed-out waiter leaves the
 * queue and the pass re-runs; placement is address-ordered first fit over
 * free extents with coalescing, granule-rounded requests, and a request is
 * served only if it both count-fits and can be placed.
 *
 * Deliberately simple: arrays, a binary heap for events, linear scans.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ST_PENDING = 0, ST_QUEUED = 1, ST_RUNNING = 2, ST_DONE = 3, ST_TIMEOUT = 4, ST_TOO_LARGE = 5 };
enum { POL_FIFO = 0, POL_FIRST_FIT = 1, POL_PRIO_FIFO = 2, POL_PRIO_FIRST_FIT = 3 };
enum { EV_COMPLETE = 0, EV_ARRIVE = 1, EV_TIMEOUT = 2 };
enum { FLAG_FIFO_BYPASS = 1 };

typedef struct {
    int32_t status;
    int32_t pad;
    int64_t grant_seq;
    uint64_t grant_t;
    uint64_t offset;
    uint64_t done_t;
} des_out;

typedef struct {
    uint64_t peak_used;
    uint64_t frag_waits;     /* passes that ended blocked by fragmentation (see policy_pass) */
    uint64_t passes;
    uint64_t makespan;       /* last done - first arrival over granted jobs */
} des_stats;

typedef struct { uint64_t t; int32_t type; int32_t id; } ev_t;

static int ev_less(const ev_t* a, const ev_t* b) {
    if (a->t != b->t) return a->t < b->t;
    if (a->type != b->type) return a->type < b->type;
    return a->id < b->id;
}

typedef struct { ev_t* v; int n, cap; } heap_t;

static void heap_push(heap_t* h, ev_t e) {
    int i = h->n++;
    h->v[i] = e;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!ev_less(&h->v[i], &h->v[p])) break;
        ev_t t = h->v[i]; h->v[i] = h->v[p]; h->v[p] = t;
        i = p;
    }
}

static ev_t heap_pop(heap_t* h) {
    ev_t top = h->v[0];
    h->v[0] = h->v[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && ev_less(&h->v[l], &h->v[m])) m = l;
        if (r < h->n && ev_less(&h->v[r], &h->v[m])) m = r;
        if (m == i) break;
        ev_t t = h->v[i]; h->v[i] = h->v[m]; h->v[m] = t;
        i = m;
    }
    return top;
}

/* Free extents of the pool, sorted by offset, never adjacent (coalesced). */
typedef struct { uint64_t* off; uint64_t* len; int n; } extents_t;

static int ext_alloc(extents_t* x, uint64_t size, uint64_t* out_off) {
    for (int i = 0; i < x->n; i++) {
        if (x->len[i] >= size) {
            *out_off = x->off[i];
            x->off[i] += size;
            x->len[i] -= size;
            if (x->len[i] == 0) {
                for (int k = i; k + 1 < x->n; k++) { x->off[k] = x->off[k + 1]; x->len[k] = x->len[k + 1]; }
                x->n--;
            }
            return 1;
        }
    }
    return 0;
}

static void ext_free(extents_t* x, uint64_t off, uint64_t size) {
    int i = 0;
    while (i < x->n && x->off[i] < off) i++;          /* insertion point */
    for (int k = x->n; k > i; k--) { x->off[k] = x->off[k - 1]; x->len[k] = x->len[k - 1]; }
    x->off[i] = off; x->len[i] = size; x->n++;
    if (i + 1 < x->n && x->off[i] + x->len[i] == x->off[i + 1]) {   /* merge right */
        x->len[i] += x->len[i + 1];
        for (int k = i + 1; k + 1 < x->n; k++) { x->off[k] = x->off[k + 1]; x->len[k] = x->len[k + 1]; }
        x->n--;
    }
    if (i > 0 && x->off[i - 1] + x->len[i - 1] == x->off[i]) {      /* merge left */
        x->len[i - 1] += x->len[i];
        for (int k = i; k + 1 < x->n; k++) { x->off[k] = x->off[k + 1]; x->len[k] = x->len[k + 1]; }
        x->n--;
    }
}

typedef struct {
    int n;
    const uint64_t *arrival, *need, *duration, *timeout;
    const int32_t* prio;
    uint64_t budget, granule;
    int policy, flags;
    uint64_t used;
    int64_t seq;
    uint64_t* need_g;
    int* q; int qn;            /* waiting job ids, in service order */
    extents_t ext;
    heap_t ev;
    des_out* out;
    des_stats* st;
} sim_t;

static int try_grant(sim_t* s, int j, uint64_t t) {
    uint64_t g = s->need_g[j];
    if (g > s->budget - s->used) return 0;                /* count test */
    uint64_t off;
    if (!ext_alloc(&s->ext, g, &off)) return 0;       /* fits the count, no extent holds it */
    s->used += g;
    if (s->used > s->st->peak_used) s->st->peak_used = s->used;
    s->out[j].status = ST_RUNNING;
    s->out[j].grant_seq = s->seq++;
    s->out[j].grant_t = t;
    s->out[j].offset = off;
    if (s->duration) {                                 /* trace mode: completion at grant + duration */
        ev_t e = { t + s->duration[j], EV_COMPLETE, j };
        heap_push(&s->ev, e);
    }
    return 1;
}

static void q_remove_at(sim_t* s, int i) {
    for (int k = i; k + 1 < s->qn; k++) s->q[k] = s->q[k + 1];
    s->qn--;
}

static void q_insert(sim_t* s, int j) {
    int pos = s->qn;
    if (s->policy == POL_PRIO_FIFO || s->policy == POL_PRIO_FIRST_FIT) {
        /* stable: after every waiter whose priority value is <= j's */
        pos = 0;
        while (pos < s->qn && s->prio[s->q[pos]] <= s->prio[j]) pos++;
    }
    for (int k = s->qn; k > pos; k--) s->q[k] = s->q[k - 1];
    s->q[pos] = j;
    s->qn++;
    s->out[j].status = ST_QUEUED;
}

static int count_fits(const sim_t* s, int j) { return s->need_g[j] <= s->budget - s->used; }

/* A pass ends blocked by fragmentation when a waiter the policy would serve
 * next fits the free byte count but no free extent can hold it: the head
 * under FIFO and Priority FIFO, any waiter under first fit, any waiter of
 * the top class under Priority MMU. */
static int blocked_by_fragmentation(const sim_t* s) {
    if (s->qn == 0) return 0;
    if (s->policy == POL_FIFO || s->policy == POL_PRIO_FIFO) return count_fits(s, s->q[0]);
    for (int i = 0; i < s->qn; i++) {
        if (s->policy == POL_PRIO_FIRST_FIT && s->prio[s->q[i]] != s->prio[s->q[0]]) break;
        if (count_fits(s, s->q[i])) return 1;
    }
    return 0;
}

/* One notification pass over the waiting queue at time t. */
static void policy_pass(sim_t* s, uint64_t t) {
    s->st->passes++;
    if (s->policy == POL_FIFO || s->policy == POL_PRIO_FIFO) {
        /* serve the head while it fits; stop at the first that does not */
        while (s->qn > 0 && try_grant(s, s->q[0], t)) q_remove_at(s, 0);
    } else if (s->policy == POL_FIRST_FIT) {
        /* serve every waiter that fits, in queue order; the others keep waiting */
        int i = 0;
        while (i < s->qn) {
            if (try_grant(s, s->q[i], t)) q_remove_at(s, i);
            else i++;
        }
    } else {
        /* first fit within the highest-priority class present; a lower class
         * is considered only once every waiter of the higher class is served */
        while (s->qn > 0) {
            int32_t p = s->prio[s->q[0]];
            int i = 0;
            while (i < s->qn && s->prio[s->q[i]] == p) {
                if (try_grant(s, s->q[i], t)) q_remove_at(s, i);
                else i++;
            }
            if (s->qn > 0 && s->prio[s->q[0]] == p) break;   /* class not emptied */
        }
    }
    if (blocked_by_fragmentation(s)) s->st->frag_waits++;
}

int des_run(int n, const uint64_t* arrival, const uint64_t* need, const uint64_t* duration,
            const uint64_t* timeout, const int32_t* prio, uint64_t budget, uint64_t granule,
            int policy, int flags, des_out* out, des_stats* st) {
    if (n < 0 || granule == 0 || policy < 0 || policy > 3) return -1;
    sim_t s;
    memset(&s, 0, sizeof s);
    memset(st, 0, sizeof *st);
    s.n = n; s.arrival = arrival; s.need = need; s.duration = duration; s.timeout = timeout;
    s.prio = prio; s.granule = granule; s.policy = policy; s.flags = flags; s.out = out; s.st = st;
    s.budget = budget / granule * granule;
    s.need_g = (uint64_t*)malloc(sizeof(uint64_t) * (n + 1));
    s.q = (int*)malloc(sizeof(int) * (n + 1));
    s.ext.off = (uint64_t*)malloc(sizeof(uint64_t) * (n + 2));
    s.ext.len = (uint64_t*)malloc(sizeof(uint64_t) * (n + 2));
    s.ev.cap = 3 * n + 1;
    s.ev.v = (ev_t*)malloc(sizeof(ev_t) * s.ev.cap);
    if (!s.need_g || !s.q || !s.ext.off || !s.ext.len || !s.ev.v) return -2;
    if (s.budget > 0) { s.ext.off[0] = 0; s.ext.len[0] = s.budget; s.ext.n = 1; }
    for (int j = 0; j < n; j++) {
        /* granule-rounded request; a request of 0 bytes still takes a granule */
        uint64_t g = (need[j] + granule - 1) / granule * granule;
        if (g == 0) g = granule;
        s.need_g[j] = g;
        out[j].status = ST_PENDING; out[j].pad = 0;
        out[j].grant_seq = -1; out[j].grant_t = 0; out[j].offset = 0; out[j].done_t = 0;
        ev_t e = { arrival[j], EV_ARRIVE, j };
        heap_push(&s.ev, e);
    }
    while (s.ev.n > 0) {
        ev_t e = heap_pop(&s.ev);
        int j = e.id;
        if (e.type == EV_COMPLETE) {
            ext_free(&s.ext, out[j].offset, s.need_g[j]);
            s.used -= s.need_g[j];
            out[j].status = ST_DONE;
            out[j].done_t = e.t;
            policy_pass(&s, e.t);
        } else if (e.type == EV_ARRIVE) {
            if (s.need_g[j] > s.budget) { out[j].status = ST_TOO_LARGE; continue; }
            if ((s.flags & FLAG_FIFO_BYPASS) && s.policy == POL_FIFO && try_grant(&s, j, e.t))
                continue;
            q_insert(&s, j);
            if (timeout[j] != UINT64_MAX) {
                uint64_t tt = arrival[j] + timeout[j];
                if (tt < arrival[j]) tt = UINT64_MAX;          /* saturate */
                ev_t te = { tt, EV_TIMEOUT, j };
                heap_push(&s.ev, te);
            }
            policy_pass(&s, e.t);
        } else { /* EV_TIMEOUT */
            if (out[j].status != ST_QUEUED) continue;
            for (int i = 0; i < s.qn; i++) if (s.q[i] == j) { q_remove_at(&s, i); break; }
            out[j].status = ST_TIMEOUT;
            out[j].done_t = e.t;
            policy_pass(&s, e.t);
        }
    }
    uint64_t first = UINT64_MAX, last = 0;
    for (int j = 0; j < n; j++) {
        if (out[j].status != ST_DONE) continue;
        if (arrival[j] < first) first = arrival[j];
        if (out[j].done_t > last) last = out[j].done_t;
    }
    st->makespan = (first == UINT64_MAX) ? 0 : last - first;
    free(s.need_g); free(s.q); free(s.ext.off); free(s.ext.len); free(s.ev.v);
    return 0;
}

/* ------------------------------------------------------------------------
 * Op-sequence mode: the life-cycle calls of Sec. IV issued one at a time by
 * clients, instead of a trace whose completions follow declared durations.
 *
 *   DECLARE(need, prio)  pre-allocation (preCudaMalloc): a request larger
 *                        than the pool is refused at once and gets no
 *                        ticket; otherwise the next ticket number is handed
 *                        out, the request joins the queue (or, under
 *                        FLAG_FIFO_BYPASS and FIFO, is served at once if it
 *                        fits) and the policy pass runs.
 *   RELEASE(ticket, b)   post-free (postCudaFree) of b declared bytes. b = 0,
 *                        or b at least the bytes the ticket still holds,
 *                        frees all of it and ends the ticket. A smaller b
 *                        shrinks the grant: the ticket keeps the first
 *                        (held - b) bytes, rounded up to the granule, at the
 *                        front of its extent, and the rest goes back to the
 *                        free list. The notification pass runs either way.
 *                        A ticket that holds nothing is refused (RC_INVALID),
 *                        and so is a second release after a full one.
 *   CANCEL(ticket)       the expiry of a blocking wait: a waiting ticket
 *                        leaves the queue (RC_TIMEOUT) and the pass re-runs;
 *                        a granted one reports RC_OK, a withdrawn one
 *                        RC_TIMEOUT again, a finished one RC_INVALID.
 *
 * After every op the scalar state is recorded (used and peak bytes, grants,
 * passes, fragmentation-blocked passes, the free extents and the largest,
 * waiting and finished tickets), so a run can be compared step by step.
 */
enum { OP_DECLARE = 0, OP_RELEASE = 1, OP_CANCEL = 2 };
enum { RC_OK = 0, RC_NOT_READY = 1, RC_TIMEOUT = 2, RC_TOO_LARGE = 3, RC_INVALID = 4 };

typedef struct {
    uint64_t t;              /* logical time of the call */
    int32_t type;            /* OP_* */
    int32_t ticket;          /* RELEASE / CANCEL: the ticket */
    uint64_t arg;            /* DECLARE: need in bytes; RELEASE: bytes freed (0 = all) */
    int32_t prio;            /* DECLARE: priority (smaller = higher) */
    int32_t pad;
} des_op;

typedef struct {
    int32_t rc;              /* RC_* */
    int32_t ticket;          /* DECLARE: ticket handed out, -1 if refused */
    uint64_t used, peak_used, grants, passes, frag_waits, max_free_extent;
    uint32_t free_extents, waiting, done, pad;
} des_op_out;

/* outcome of a single op on the simulator state (see the comment above) */
static int32_t op_step(sim_t* s, const des_op* op, int* n_tickets, uint64_t* raw, int32_t* prio,
                       int32_t* ticket_out) {
    *ticket_out = -1;
    if (op->type == OP_DECLARE) {
        uint64_t g = (op->arg + s->granule - 1) / s->granule * s->granule;
        if (g == 0) g = s->granule;
        if (g > s->budget) return RC_TOO_LARGE;
        int j = (*n_tickets)++;
        *ticket_out = j;
        s->need_g[j] = g;
        raw[j] = op->arg;
        prio[j] = op->prio;
        s->out[j].status = ST_PENDING;
        s->out[j].grant_seq = -1;
        if ((s->flags & FLAG_FIFO_BYPASS) && s->policy == POL_FIFO && try_grant(s, j, op->t))
            return RC_OK;
        q_insert(s, j);
        policy_pass(s, op->t);
        return RC_OK;
    }
    int j = op->ticket;
    if (j < 0 || j >= *n_tickets) return RC_INVALID;
    if (op->type == OP_RELEASE) {
        if (s->out[j].status != ST_RUNNING) return RC_INVALID;
        if (op->arg == 0 || op->arg >= raw[j]) {
            ext_free(&s->ext, s->out[j].offset, s->need_g[j]);
            s->used -= s->need_g[j];
            s->out[j].status = ST_DONE;
            s->out[j].done_t = op->t;
        } else {
            uint64_t keep_raw = raw[j] - op->arg;
            uint64_t keep = (keep_raw + s->granule - 1) / s->granule * s->granule;
            uint64_t freed = s->need_g[j] - keep;
            if (freed > 0) ext_free(&s->ext, s->out[j].offset + keep, freed);
            s->used -= freed;
            s->need_g[j] = keep;
            raw[j] = keep_raw;
        }
        policy_pass(s, op->t);
        return RC_OK;
    }
    if (op->type == OP_CANCEL) {
        int32_t st = s->out[j].status;
        if (st == ST_RUNNING) return RC_OK;
        if (st == ST_TIMEOUT) return RC_TIMEOUT;
        if (st != ST_QUEUED) return RC_INVALID;
        for (int i = 0; i < s->qn; i++) if (s->q[i] == j) { q_remove_at(s, i); break; }
        s->out[j].status = ST_TIMEOUT;
        s->out[j].done_t = op->t;
        policy_pass(s, op->t);
        return RC_TIMEOUT;
    }
    return RC_INVALID;
}

/* Run n_ops life-cycle calls; tickets[] gets one record per ticket handed out
 * (at most n_ops), ops_out[] one state record per op; *n_tickets_out the
 * number of tickets. Returns 0, or a negative value on bad arguments. */
int des_ops_run(int n_ops, const des_op* ops, uint64_t budget, uint64_t granule, int policy, int flags,
                des_out* tickets, des_op_out* ops_out, int* n_tickets_out) {
    if (n_ops < 0 || granule == 0 || policy < 0 || policy > 3) return -1;
    sim_t s;
    des_stats st;
    memset(&s, 0, sizeof s);
    memset(&st, 0, sizeof st);
    int cap = n_ops + 1;
    s.granule = granule; s.policy = policy; s.flags = flags; s.out = tickets; s.st = &st;
    s.budget = budget / granule * granule;
    s.duration = NULL;
    uint64_t* raw = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    int32_t* prio = (int32_t*)malloc(sizeof(int32_t) * cap);
    s.prio = prio;
    s.need_g = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    s.q = (int*)malloc(sizeof(int) * cap);
    s.ext.off = (uint64_t*)malloc(sizeof(uint64_t) * (cap + 2));
    s.ext.len = (uint64_t*)malloc(sizeof(uint64_t) * (cap + 2));
    if (!raw || !prio || !s.need_g || !s.q || !s.ext.off || !s.ext.len) return -2;
    if (s.budget > 0) { s.ext.off[0] = 0; s.ext.len[0] = s.budget; s.ext.n = 1; }
    for (int j = 0; j < n_ops; j++) {
        tickets[j].status = ST_PENDING; tickets[j].pad = 0; tickets[j].grant_seq = -1;
        tickets[j].grant_t = 0; tickets[j].offset = 0; tickets[j].done_t = 0;
    }
    int n_tickets = 0;
    for (int k = 0; k < n_ops; k++) {
        des_op_out* o = &ops_out[k];
        memset(o, 0, sizeof *o);
        o->rc = op_step(&s, &ops[k], &n_tickets, raw, prio, &o->ticket);
        o->used = s.used;
        o->peak_used = st.peak_used;
        o->grants = (uint64_t)s.seq;
        o->passes = st.passes;
        o->frag_waits = st.frag_waits;
        o->free_extents = (uint32_t)s.ext.n;
        for (int i = 0; i < s.ext.n; i++)
            if (s.ext.len[i] > o->max_free_extent) o->max_free_extent = s.ext.len[i];
        o->waiting = (uint32_t)s.qn;
        for (int j = 0; j < n_tickets; j++)
            if (tickets[j].status == ST_DONE || tickets[j].status == ST_TIMEOUT) o->done++;
    }
    *n_tickets_out = n_tickets;
    free(raw); free(prio); free(s.need_g); free(s.q); free(s.ext.off); free(s.ext.len);
    return 0;
}
