// mb_server.cu -- continuous-batching request loop on top of the batch API.
//
// Requests (one simulation each: grid, body, motion, initial state, number of
// CFL steps) queue on submission.  Every tick admits queued requests while
// the device-memory budget and the slot limit allow, advances every admitted
// simulation by one time step in the batch's shared launches, and retires the
// simulations that reached their step count: their final state is copied to
// the caller's buffer and their device memory released, which lets the next
// requests in.  States stay resident on the device from admission to
// retirement.  Admission happens only when the batch has taken an even number
// of steps, so every simulation sweeps x,y / y,x in the same order as it would
// alone (the order alternates with the step count).
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/mb.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    mb_grid grid;
    double gamma;
    mb_motion motion;
    int npoly;
    std::vector<int> pstart, pmov;
    std::vector<double> vx, vy;
    std::vector<double> Q0;
    double t0;
    int nsteps;
    double *Qout;
    int state = 0;            // 0 queued, 1 running, 2 done, < 0 failed (mb_status)
    double t_submit = 0, t_admit = 0, t_done = 0;
    int steps_done = 0;
    size_t bytes = 0;
    std::string error;        // why it failed
    mb_body body() const {
        mb_body b;
        b.npoly = npoly;
        b.poly_start = pstart.data();
        b.poly_moving = pmov.data();
        b.vx = vx.data();
        b.vy = vy.data();
        return b;
    }
};

}  // namespace

struct mb_server {
    int precision, equation, max_active;
    double budget;
    double used = 0.0;
    mb_sim *sim = nullptr;
    long long batch_steps = 0;        // steps of the batch since it was last empty
    std::vector<Request> req;
    std::deque<int> queue;
    std::vector<int> active;          // request id of each batch instance, in instance order
    int n_done = 0;
    std::string err;
};

static mb_status srv_fail(mb_server *s, mb_status st, const std::string &m) {
    s->err = m;
    return st;
}

extern "C" {

mb_status mb_server_create(int precision, int equation, double budget_bytes, int max_active, mb_server **out) {
    if (!out) return MB_E_INVAL;
    *out = nullptr;
    if ((precision != MB_FP32 && precision != MB_FP64) || (equation != MB_EULER && equation != MB_ADVECTION) ||
        !(budget_bytes > 0.0) || max_active < 1)
        return MB_E_INVAL;
    mb_server *s = new mb_server();
    s->precision = precision;
    s->equation = equation;
    s->budget = budget_bytes;
    s->max_active = max_active;
    *out = s;
    return MB_OK;
}

void mb_server_destroy(mb_server *srv) {
    if (!srv) return;
    if (srv->sim) mb_destroy(srv->sim);
    delete srv;
}

const char *mb_server_last_error(const mb_server *srv) { return srv ? srv->err.c_str() : ""; }

mb_status mb_server_submit(mb_server *srv, const mb_request *r, int *id) {
    if (!srv || !r || !r->Q0 || r->nsteps < 0) return MB_E_INVAL;
    const int req_eq = r->grid.equation == MB_EULER_AXISYM ? MB_EULER : r->grid.equation;
    if (r->grid.precision != srv->precision || req_eq != srv->equation)
        return srv_fail(srv, MB_E_INVAL, "request precision or equation differs from the server's");
    const mb_body &b = r->body;
    if (b.npoly < 0 || (b.npoly > 0 && (!b.poly_start || !b.poly_moving || !b.vx || !b.vy)))
        return srv_fail(srv, MB_E_INVAL, "bad body");
    Request q;
    q.grid = r->grid;
    q.gamma = r->gamma;
    q.motion = r->motion;
    q.npoly = b.npoly;
    if (b.npoly > 0) {
        q.pstart.assign(b.poly_start, b.poly_start + b.npoly + 1);
        q.pmov.assign(b.poly_moving, b.poly_moving + b.npoly);
        const int nv = b.poly_start[b.npoly];
        q.vx.assign(b.vx, b.vx + nv);
        q.vy.assign(b.vy, b.vy + nv);
    } else {
        q.pstart.assign(1, 0);
        q.pmov.assign(1, 0);
    }
    const int nc = req_eq == MB_EULER ? 4 : 1;
    q.Q0.assign(r->Q0, r->Q0 + (size_t)nc * r->grid.nx * r->grid.ny);
    q.t0 = r->t0;
    q.nsteps = r->nsteps;
    q.Qout = r->Qout;
    q.t_submit = now_s();
    srv->req.push_back(std::move(q));
    const int k = (int)srv->req.size() - 1;
    srv->queue.push_back(k);
    if (id) *id = k;
    return MB_OK;
}

// admit the request at the head of the queue; returns false when it does not
// fit (budget or slots) and it should wait
static bool admit_one(mb_server *srv, mb_status *st) {
    *st = MB_OK;
    const int k = srv->queue.front();
    Request &q = srv->req[k];
    if ((int)srv->active.size() >= srv->max_active) return false;
    const mb_body body = q.body();
    q.bytes = mb_request_bytes(&q.grid, &body, &q.motion);
    // wait for memory unless nothing else is running (a request larger than
    // the whole budget runs alone)
    if (!srv->active.empty() && srv->used + (double)q.bytes > srv->budget) return false;
    int inst = -1;
    mb_status r;
    if (!srv->sim) {
        r = mb_create(&q.grid, q.gamma, &body, &q.motion, &srv->sim);
        inst = 0;
        if (r != MB_OK) {
            srv->sim = nullptr;
            q.state = r;
            srv->queue.pop_front();
            srv->err = mb_last_error(nullptr);
            q.error = srv->err;
            ++srv->n_done;
            return true;
        }
    } else {
        r = mb_batch_add(srv->sim, &q.grid, q.gamma, &body, &q.motion, &inst);
        if (r != MB_OK) {
            q.state = r;
            srv->queue.pop_front();
            srv->err = mb_last_error(srv->sim);
            q.error = srv->err;
            ++srv->n_done;
            return true;
        }
    }
    r = mb_write_state(srv->sim, inst, q.Q0.data(), q.t0);
    if (r != MB_OK) {
        *st = r;
        srv->err = mb_last_error(srv->sim);
        return false;
    }
    srv->used += (double)q.bytes;
    q.state = 1;
    q.t_admit = now_s();
    q.Q0.clear();
    q.Q0.shrink_to_fit();
    srv->active.push_back(k);
    srv->queue.pop_front();
    return true;
}

mb_status mb_server_tick(mb_server *srv, int *n_active, int *n_queued, int *n_done) {
    if (!srv) return MB_E_INVAL;
    mb_status st = MB_OK;
    // 1. admission at even batch steps (a new simulation starts with the
    //    batch's sweep order)
    if (srv->active.empty()) srv->batch_steps = 0;
    if (srv->batch_steps % 2 == 0) {
        while (!srv->queue.empty()) {
            if (!admit_one(srv, &st)) break;
        }
        if (st != MB_OK) return st;
    }
    // 2. one time step of every admitted simulation
    if (!srv->active.empty()) {
        st = mb_run(srv->sim, 1, 0.0);
        if (st != MB_OK) return srv_fail(srv, st, mb_last_error(srv->sim));
        ++srv->batch_steps;
        for (int k : srv->active) ++srv->req[k].steps_done;
    }
    // 3. retirement of the simulations that reached their step count
    for (int pos = (int)srv->active.size() - 1; pos >= 0; --pos) {
        Request &q = srv->req[srv->active[pos]];
        if (q.steps_done < q.nsteps) continue;
        st = mb_read_state(srv->sim, pos, q.Qout, nullptr, nullptr);
        q.state = st == MB_OK ? 2 : st;
        if (st != MB_OK) q.error = mb_last_error(srv->sim);
        q.t_done = now_s();
        mb_status r = mb_batch_remove(srv->sim, pos);
        if (r != MB_OK) return srv_fail(srv, r, mb_last_error(srv->sim));
        srv->used -= (double)q.bytes;
        srv->active.erase(srv->active.begin() + pos);
        ++srv->n_done;
    }
    if (srv->active.empty()) srv->batch_steps = 0;
    if (n_active) *n_active = (int)srv->active.size();
    if (n_queued) *n_queued = (int)srv->queue.size();
    if (n_done) *n_done = srv->n_done;
    return MB_OK;
}

const char *mb_server_request_error(const mb_server *srv, int id) {
    if (!srv || id < 0 || id >= (int)srv->req.size()) return "";
    return srv->req[id].error.c_str();
}

mb_status mb_server_query(mb_server *srv, int id, int *state, double *info) {
    if (!srv || id < 0 || id >= (int)srv->req.size()) return MB_E_INVAL;
    const Request &q = srv->req[id];
    if (state) *state = q.state;
    if (info) {
        info[0] = q.t_submit;
        info[1] = q.t_admit;
        info[2] = q.t_done;
        info[3] = (double)q.steps_done;
        info[4] = (double)q.bytes;
    }
    return MB_OK;
}

}  // extern "C"
