// serve.cu -- continuous-batching server for encrypted inference requests.
//
// A model is a program over a request's registers (register 0 holds the
// input and, at the end, the output): a step applies a prepared layer
// (bootstraps included), adds two registers at a level, or multiplies one by
// a constant rescaled onto the model's scale.  A chain of layers is the
// program of one layer step per layer on register 0; a residual network uses
// more registers.  Requests of one or more models on one context (evaluation
// keys resident) arrive over time.  A request is admitted while fewer than
// `max_active` are in flight and the device has at least `min_free` bytes
// free; the rest wait in arrival order.  Each scheduling step takes the
// oldest admitted request's stage (model, next step), runs that step for
// every admitted request at the same stage -- a layer step as one batch
// (fheon_layer_apply_batch: their rotations share launches) -- and advances
// them; requests past their model's last step are done and keep their result
// until it is taken.  A request's result is the one the model gives its input
// alone, bit for bit: batching changes launches, never arithmetic.  With an
// admission timeout, a request still waiting that long after its submission
// is dropped at the next admission and its result reports FHEON_ERR_TIMEOUT.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "layer.h"

using namespace fheon;

struct fheon_model {
    fheon_ctx *ctx = nullptr;
    std::vector<fheon_step> steps;
    u32 nreg = 1;
    double scale = 0; // target of constant steps
};

namespace {
struct Request {
    uint64_t id = 0, seq = 0;
    const fheon_model *model = nullptr;
    u32 next = 0;                 // next step
    std::vector<fheon_ct *> reg;  // registers
    fheon_ct *nxt = nullptr, *aux = nullptr; // a step's output and an operand copy
    bool done = false;
    int status = FHEON_OK; // FHEON_ERR_TIMEOUT: dropped before admission
    std::chrono::steady_clock::time_point submitted;
    ~Request()
    {
        for (fheon_ct *c : reg) fheon_ct_destroy(c);
        fheon_ct_destroy(nxt);
        fheon_ct_destroy(aux);
    }
};

// one non-layer step of one request: its output into r->nxt
int run_step(fheon_ctx *ctx, const fheon_model *m, const fheon_step &st, Request *r)
{
    int rc;
    if (st.op == FHEON_STEP_ADD) {
        if ((rc = fheon_drop_level(ctx, r->reg[st.src], st.level, r->aux))) return rc;
        if ((rc = fheon_drop_level(ctx, r->reg[st.src2], st.level, r->nxt))) return rc;
        return fheon_add(ctx, r->aux, r->nxt, r->nxt);
    }
    return fheon_mul_const_rescale(ctx, r->reg[st.src], st.c, m->scale, r->nxt);
}
} // namespace

struct fheon_server {
    fheon_ctx *ctx = nullptr;
    u32 max_active = 1;
    size_t min_free = 0;
    std::deque<Request *> waiting;
    std::vector<Request *> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_id = 1, next_seq = 0, steps = 0;
    u32 max_batch = 0;
    double admit_timeout = 0; // seconds a request may wait for admission; 0: no limit
};

namespace {
// drop the waiting requests past the admission timeout (counted in *expired),
// then admit what fits
int admit(fheon_server *s, u32 *expired)
{
    if (s->admit_timeout > 0) {
        const auto now = std::chrono::steady_clock::now();
        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
            Request *r = *it;
            if (std::chrono::duration<double>(now - r->submitted).count() > s->admit_timeout) {
                r->done = true;
                r->status = FHEON_ERR_TIMEOUT;
                ++*expired;
                it = s->waiting.erase(it);
            } else {
                ++it;
            }
        }
    }
    while (!s->waiting.empty() && s->active.size() < s->max_active) {
        if (s->min_free) {
            size_t free_b = 0, total_b = 0;
            FHEON_CUDA(s->ctx, cudaMemGetInfo(&free_b, &total_b));
            if (free_b < s->min_free && !s->active.empty()) break; // the oldest always gets in
        }
        Request *r = s->waiting.front();
        s->waiting.pop_front();
        r->seq = s->next_seq++;
        s->active.push_back(r);
    }
    return FHEON_OK;
}
} // namespace

extern "C" {

int fheon_model_create_program(fheon_ctx *ctx, const fheon_step *steps, uint32_t n, uint32_t nreg, double scale,
                               fheon_model **out)
{
    if (!ctx || !out || !n || !steps || !nreg || nreg > 64) return FHEON_ERR_ARG;
    for (u32 i = 0; i < n; i++) {
        const fheon_step &st = steps[i];
        const bool regs_ok = st.src < nreg && st.dst < nreg && (st.op != FHEON_STEP_ADD || st.src2 < nreg);
        if (!regs_ok) return fail(ctx, FHEON_ERR_ARG, "model step %u: register out of range", i);
        if (st.op == FHEON_STEP_LAYER && !st.layer) return fail(ctx, FHEON_ERR_ARG, "model step %u: no layer", i);
        if (st.op == FHEON_STEP_ADD && st.level < 1) return fail(ctx, FHEON_ERR_ARG, "model step %u: level 0", i);
        if (st.op == FHEON_STEP_SCALE && !(scale > 0)) return fail(ctx, FHEON_ERR_ARG, "model step %u: no scale", i);
        if (st.op > FHEON_STEP_SCALE) return fail(ctx, FHEON_ERR_ARG, "model step %u: unknown op %u", i, st.op);
    }
    fheon_model *m = new fheon_model();
    m->ctx = ctx;
    m->steps.assign(steps, steps + n);
    m->nreg = nreg;
    m->scale = scale;
    *out = m;
    return FHEON_OK;
}

int fheon_model_create(fheon_ctx *ctx, const fheon_layer *const *layers, uint32_t n, fheon_model **out)
{
    if (!ctx || !out || !n || !layers) return FHEON_ERR_ARG;
    std::vector<fheon_step> st(n);
    for (u32 i = 0; i < n; i++) {
        if (!layers[i]) return FHEON_ERR_ARG;
        st[i] = fheon_step{FHEON_STEP_LAYER, 0, 0, 0, 0, layers[i], 0.0};
    }
    return fheon_model_create_program(ctx, st.data(), n, 1, 0.0, out);
}

int fheon_model_run(fheon_ctx *ctx, const fheon_model *m, const fheon_ct *in, fheon_ct *out)
{
    if (!ctx || !m || !in || !out || m->ctx != ctx) return FHEON_ERR_ARG;
    Request r;
    r.model = m;
    r.reg.assign(m->nreg, nullptr);
    int rc;
    for (fheon_ct *&c : r.reg)
        if ((rc = fheon_ct_create(ctx, in->level, in->scale, &c))) return rc;
    if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r.nxt))) return rc;
    if ((rc = fheon_ct_create(ctx, in->level, in->scale, &r.aux))) return rc;
    if ((rc = fheon_drop_level(ctx, in, in->level, r.reg[0]))) return rc;
    for (const fheon_step &st : m->steps) {
        if (st.op == FHEON_STEP_LAYER) {
            if ((rc = fheon_layer_apply(ctx, st.layer, r.reg[st.src], r.nxt))) return rc;
        } else if ((rc = run_step(ctx, m, st, &r))) {
            return rc;
        }
        std::swap(r.reg[st.dst], r.nxt);
    }
    rc = fheon_drop_level(ctx, r.reg[0], r.reg[0]->level, out);
    if (!rc) rc = fheon_sync(ctx); // the request's buffers go with it
    return rc;
}

int fheon_model_destroy(fheon_model *m)
{
    delete m;
    return FHEON_OK;
}

int fheon_server_create(fheon_ctx *ctx, uint32_t max_active, size_t min_free, fheon_server **out)
{
    if (!ctx || !out || !max_active) return FHEON_ERR_ARG;
    fheon_server *s = new fheon_server();
    s->ctx = ctx;
    s->max_active = max_active;
    s->min_free = min_free;
    *out = s;
    return FHEON_OK;
}

int fheon_server_destroy(fheon_server *s)
{
    if (s && s->ctx) cudaStreamSynchronize(s->ctx->stream);
    delete s;
    return FHEON_OK;
}

int fheon_server_submit(fheon_server *s, const fheon_model *m, const fheon_ct *in, uint64_t *id)
{
    if (!s || !m || !in || !id || m->ctx != s->ctx) return FHEON_ERR_ARG;
    std::unique_ptr<Request> r(new Request());
    int rc;
    r->reg.assign(m->nreg, nullptr);
    for (fheon_ct *&c : r->reg)
        if ((rc = fheon_ct_create(s->ctx, in->level, in->scale, &c))) return rc;
    if ((rc = fheon_ct_create(s->ctx, in->level, in->scale, &r->nxt))) return rc;
    if ((rc = fheon_ct_create(s->ctx, in->level, in->scale, &r->aux))) return rc;
    if ((rc = fheon_drop_level(s->ctx, in, in->level, r->reg[0]))) return rc; // the request's own copy
    r->id = s->next_id++;
    r->model = m;
    r->submitted = std::chrono::steady_clock::now();
    *id = r->id;
    s->waiting.push_back(r.get());
    s->all.emplace(r->id, std::move(r));
    return FHEON_OK;
}

int fheon_server_step(fheon_server *s, uint32_t *n_done)
{
    if (!s) return FHEON_ERR_ARG;
    Range range("server_step");
    if (n_done) *n_done = 0;
    u32 expired = 0;
    int rc = admit(s, &expired);
    if (n_done) *n_done = expired;
    if (rc) return rc;
    if (s->active.empty()) return FHEON_OK;
    const Request *oldest = *std::min_element(s->active.begin(), s->active.end(),
                                              [](const Request *a, const Request *b) { return a->seq < b->seq; });
    const fheon_model *m = oldest->model;
    const u32 stage = oldest->next;
    std::vector<Request *> batch;
    for (Request *r : s->active)
        if (r->model == m && r->next == stage) batch.push_back(r);
    const fheon_step &st = m->steps[stage];
    if (st.op == FHEON_STEP_LAYER) {
        std::vector<const fheon_ct *> ins;
        std::vector<fheon_ct *> outs;
        for (Request *r : batch) {
            ins.push_back(r->reg[st.src]);
            outs.push_back(r->nxt);
        }
        if ((rc = fheon_layer_apply_batch(s->ctx, st.layer, ins.data(), (u32)batch.size(), outs.data()))) return rc;
    } else {
        for (Request *r : batch)
            if ((rc = run_step(s->ctx, m, st, r))) return rc;
    }
    s->steps++;
    s->max_batch = std::max<u32>(s->max_batch, (u32)batch.size());
    u32 done = 0;
    for (Request *r : batch) {
        std::swap(r->reg[st.dst], r->nxt);
        r->next++;
        if (r->next == m->steps.size()) {
            r->done = true;
            done++;
        }
    }
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](const Request *r) { return r->done; }),
                    s->active.end());
    if ((rc = fheon_sync(s->ctx))) return rc;
    if (n_done) *n_done = done + expired;
    return FHEON_OK;
}

int fheon_server_result(fheon_server *s, uint64_t id, fheon_ct *out)
{
    if (!s || !out) return FHEON_ERR_ARG;
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(s->ctx, FHEON_ERR_ARG, "no request %llu", (unsigned long long)id);
    if (it->second->status != FHEON_OK) {
        const int st = it->second->status;
        s->all.erase(it);
        return fail(s->ctx, st, "request %llu waited longer than the admission timeout", (unsigned long long)id);
    }
    if (!it->second->done) return FHEON_PENDING;
    const fheon_ct *r = it->second->reg[0];
    int rc = fheon_drop_level(s->ctx, r, r->level, out);
    if (rc) return rc;
    if ((rc = fheon_sync(s->ctx))) return rc;
    s->all.erase(it);
    return FHEON_OK;
}

int fheon_server_set_admit_timeout(fheon_server *s, double seconds)
{
    if (!s || !(seconds >= 0) || std::isinf(seconds)) return FHEON_ERR_ARG;
    s->admit_timeout = seconds;
    return FHEON_OK;
}

int fheon_server_stats(const fheon_server *s, uint64_t *steps, uint32_t *max_batch, uint32_t *active,
                       uint32_t *waiting)
{
    if (!s) return FHEON_ERR_ARG;
    if (steps) *steps = s->steps;
    if (max_batch) *max_batch = s->max_batch;
    if (active) *active = (uint32_t)s->active.size();
    if (waiting) *waiting = (uint32_t)s->waiting.size();
    return FHEON_OK;
}

} // extern "C"
