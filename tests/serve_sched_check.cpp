// Host check of the serving admission policy (paper_2607_23187_b300/csrc/
// serve_sched.h) with stand-in lanes and requests.  Random arrivals and
// completions on random lane counts, budgets and SM caps; after every step
// the invariants of the policy are checked against a restatement of its
// rules written here.  Also replays the one-lane run order that the GPU
// test checks.  Exit status 0 when everything holds.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "serve_sched.h"

using pjac::SERVE_BATCH_MAX_N;
using pjac::SERVE_MAX_BYPASS;

struct Req {
    int n;
    int pivot;
    double tol;
    size_t footprint;
    int bypassed = 0;
    long id = 0;
    bool done = false;
};

struct Lane {
    bool busy = false;
    bool hi = false;
    int sms = 0;
    std::vector<Req*> reqs;
};

static unsigned g_seed = 0;
static int g_step = 0;

#define CHECK(c)                                                                                       \
    do {                                                                                               \
        if (!(c)) {                                                                                    \
            std::fprintf(stderr, "FAIL line %d: %s (seed %u, step %d)\n", __LINE__, #c, g_seed, g_step); \
            std::exit(1);                                                                              \
        }                                                                                              \
    } while (0)

static int sms_of(int n) { return n <= 384 ? 1 : (n <= 1024 ? 4 : 8); }

static bool fits(const pjac::ServeQueue<Req>& q, const Req* r) {
    size_t room = q.budget > q.in_use ? q.budget - q.in_use : 0;
    return r->footprint <= room || q.in_use == 0;
}

// Bookkeeping: in_use and sms_used are what the busy lanes hold.
static void check_books(const pjac::ServeQueue<Req>& q, const std::vector<Lane>& lanes) {
    size_t bytes = 0;
    int sms = 0;
    int large_running = 0;
    for (const Lane& L : lanes) {
        if (!L.busy) {
            CHECK(L.reqs.empty() && L.sms == 0);
            continue;
        }
        for (const Req* r : L.reqs) bytes += r->footprint;
        sms += L.sms;
        if (L.sms > 0) large_running++;
    }
    CHECK(bytes == q.in_use);
    CHECK(sms == q.sms_used);
    CHECK(q.sms_used <= q.sms_cap || large_running == 1);
    for (const Req* r : q.large) CHECK(r->bypassed <= SERVE_MAX_BYPASS);
}

// One admission pass, checking each admission against the rules.
static void admit_all(pjac::ServeQueue<Req>& q, std::vector<Lane>& lanes, std::vector<long>* order) {
    for (;;) {
        bool free_hi = false, free_lo = false;
        for (const Lane& L : lanes) {
            if (!L.busy && L.hi) free_hi = true;
            if (!L.busy && !L.hi) free_lo = true;
        }
        Req* small = q.small.empty() ? nullptr : q.small.front();
        Req* big = q.large.empty() ? nullptr : q.large.front();
        const bool small_ok = (free_hi || free_lo) && small && fits(q, small);
        const bool big_ok = free_lo && big && fits(q, big) &&
                            (q.sms_used == 0 || q.sms_used + sms_of(big->n) <= q.sms_cap);
        const int big_bypassed = big ? big->bypassed : 0;
        const size_t in_use_before = q.in_use;
        Lane* L = pjac::serve_admit(q, lanes, sms_of);
        if (!L) {
            // nothing admissible is left behind
            CHECK(!small_ok && !big_ok);
            return;
        }
        CHECK(!L->busy && !L->reqs.empty());
        L->busy = true;
        const Req* r0 = L->reqs[0];
        if (r0->n <= SERVE_BATCH_MAX_N) {
            // a micro-batch: the oldest small request first, the rest in
            // arrival order with its pivot rule and tolerance
            CHECK(small_ok && r0 == small);
            CHECK(!(big_ok && big_bypassed >= SERVE_MAX_BYPASS));
            CHECK(L->hi || !free_hi);
            CHECK(L->sms == 0);
            for (size_t k = 0; k < L->reqs.size(); ++k) {
                const Req* r = L->reqs[k];
                CHECK(r->n <= SERVE_BATCH_MAX_N && r->pivot == r0->pivot && r->tol == r0->tol);
                if (k) CHECK(r->id > L->reqs[k - 1]->id);
            }
            if (big_ok) CHECK(big->bypassed == big_bypassed + 1);
            // no waiting request of the same kind that fitted was left out
            size_t held = 0;
            for (const Req* r : L->reqs) held += r->footprint;
            size_t room = q.budget > in_use_before ? q.budget - in_use_before : 0;
            for (const Req* r : q.small)
                if (r->pivot == r0->pivot && r->tol == r0->tol && r->id > r0->id)
                    CHECK(held + r->footprint > room || L->reqs.size() == pjac::SERVE_MAX_BATCH);
        } else {
            // the oldest large request alone, on a low-priority lane
            CHECK(big_ok && r0 == big && L->reqs.size() == 1 && !L->hi);
            CHECK(!small_ok || big_bypassed >= SERVE_MAX_BYPASS);
            CHECK(L->sms == sms_of(r0->n));
        }
        // the budget holds, except for one request admitted onto an idle device
        CHECK(q.in_use <= q.budget || (in_use_before == 0 && L->reqs.size() == 1));
        if (order)
            for (const Req* r : L->reqs) order->push_back(r->id);
        check_books(q, lanes);
    }
}

static void finish(pjac::ServeQueue<Req>& q, Lane& L) {
    pjac::serve_release(q, L);
    for (Req* r : L.reqs) r->done = true;
    L.reqs.clear();
    L.busy = false;
}

static std::vector<Lane> make_lanes(int nl) {
    std::vector<Lane> lanes(nl);
    int n_hi = nl >= 2 ? std::max(1, nl / 8) : 0;   // as pjac_serve_create
    for (int k = 0; k < n_hi; ++k) lanes[k].hi = true;
    return lanes;
}

static void random_run(unsigned seed) {
    g_seed = seed;
    std::mt19937 rng(seed);
    auto pick = [&](int m) { return (int)(rng() % (unsigned)m); };
    const int lane_counts[] = {1, 2, 3, 4, 8, 32};
    const int sizes[] = {16, 64, 128, 256, 257, 300, 512, 1024, 2048};
    std::vector<Lane> lanes = make_lanes(lane_counts[pick(6)]);
    pjac::ServeQueue<Req> q;
    const int caps[] = {1, 4, 8, 16, 130};
    q.sms_cap = caps[pick(5)];
    const size_t unit = (size_t)256 * 256 * 80;
    const size_t budgets[] = {unit / 2, 3 * unit, 40 * unit, (size_t)1 << 40};
    q.budget = budgets[pick(4)];
    std::vector<Req*> all;
    const int steps = 3000;
    for (g_step = 0; g_step < steps || !q.small.empty() || !q.large.empty(); ++g_step) {
        CHECK(g_step < 100000);   // every request completes
        if (g_step < 2 * steps / 3 && pick(3) == 0) {
            int m = 1 + pick(3);
            for (int k = 0; k < m; ++k) {
                Req* r = new Req();
                r->n = sizes[pick(9)];
                r->pivot = pick(4) == 0 ? 1 : 0;
                r->tol = pick(5) == 0 ? 2e-15 : 1e-15;
                r->footprint = (size_t)r->n * r->n * 80;
                r->id = (long)all.size();
                all.push_back(r);
                q.push(r);
            }
        }
        if (pick(2) == 0) {
            std::vector<Lane*> busy;
            for (Lane& L : lanes)
                if (L.busy) busy.push_back(&L);
            if (!busy.empty()) finish(q, *busy[pick((int)busy.size())]);
        }
        admit_all(q, lanes, nullptr);
        check_books(q, lanes);
    }
    for (Lane& L : lanes)
        if (L.busy) finish(q, L);
    check_books(q, lanes);
    CHECK(q.in_use == 0 && q.sms_used == 0);
    for (Req* r : all) {
        CHECK(r->done);
        delete r;
    }
}

// One lane: a large request A runs; a large L and six small requests with
// distinct tolerances wait.  Run order A, S1..S4, L, S5, S6.
static void one_lane_order() {
    g_seed = 0;
    g_step = 0;
    std::vector<Lane> lanes = make_lanes(1);
    pjac::ServeQueue<Req> q;
    q.sms_cap = 130;
    q.budget = (size_t)1 << 40;
    std::vector<Req> reqs(8);
    const int ns[8] = {400, 300, 64, 80, 96, 112, 128, 144};
    for (int k = 0; k < 8; ++k) {
        reqs[k].n = ns[k];
        reqs[k].pivot = 0;
        reqs[k].tol = k < 2 ? 1e-15 : (k - 1) * 1e-15;
        reqs[k].footprint = (size_t)ns[k] * ns[k] * 80;
        reqs[k].id = k;
    }
    std::vector<long> order;
    q.push(&reqs[0]);
    admit_all(q, lanes, &order);   // A takes the lane at once
    for (int k = 1; k < 8; ++k) q.push(&reqs[k]);
    while (order.size() < 8) {
        CHECK(lanes[0].busy);
        finish(q, lanes[0]);
        admit_all(q, lanes, &order);
        g_step++;
    }
    const long want[8] = {0, 2, 3, 4, 5, 1, 6, 7};
    for (int k = 0; k < 8; ++k) CHECK(order[k] == want[k]);
}

int main(int argc, char** argv) {
    int runs = argc > 1 ? std::atoi(argv[1]) : 300;
    one_lane_order();
    for (int s = 1; s <= runs; ++s) random_run((unsigned)s);
    std::printf("ok %d runs\n", runs);
    return 0;
}
