// Admission policy of the serving form (pjac_serve_*).  Free of CUDA, so
// that host tests can drive it with stand-in lanes and requests; serve.cu
// instantiates it with its own.
//
// Requests wait in two FIFOs: small (order <= SERVE_BATCH_MAX_N) and large.
// Whenever a lane is free:
//   - small requests go first: the oldest one and every other waiting small
//     request with its pivot rule and tolerance form one micro-batch, within
//     the device-memory budget, on a free high-priority lane if there is one;
//   - otherwise the oldest large request takes a free low-priority lane
//     alone, provided the SMs of all running large requests stay within
//     sms_cap;
//   - the oldest large request is passed over by at most SERVE_MAX_BYPASS
//     micro-batches while it could have run, so small work cannot starve it.
// A request is admitted only while the bytes of admitted work stay within
// the budget; with nothing admitted, one request always is.
#pragma once
#include <algorithm>
#include <cstddef>
#include <deque>
#include <vector>

namespace pjac {

constexpr int SERVE_BATCH_MAX_N = 256;      // orders served by micro-batches
constexpr int SERVE_MAX_BYPASS = 4;         // micro-batches that may pass the oldest large request
constexpr size_t SERVE_MAX_BATCH = 4096;    // requests in one micro-batch

// Waiting requests and what admitted work holds.  Req has the fields n,
// pivot, tol, footprint (device bytes) and bypassed (an int, initially 0).
template <class Req>
struct ServeQueue {
    std::deque<Req*> small, large;   // waiting, oldest first
    size_t budget = 0;               // device bytes admitted work may hold
    size_t in_use = 0;               // device bytes admitted work holds
    int sms_cap = 0;                 // SMs running large requests may hold together
    int sms_used = 0;                // SMs running large requests hold

    void push(Req* q) { (q->n <= SERVE_BATCH_MAX_N ? small : large).push_back(q); }
    size_t waiting() const { return small.size() + large.size(); }
};

// Admits the next piece of work onto a free lane.  Lane has the fields busy,
// hi (high-priority stream), sms and reqs (a std::vector<Req*>, empty while
// the lane is free); sms_of(n) is the number of SMs a large request of order
// n holds.  Fills the chosen lane's reqs and sms, takes the requests off the
// queue and adds their bytes and SMs to in_use and sms_used; the caller
// marks the lane busy.  Returns that lane, or nullptr when nothing can be
// admitted now.
template <class Req, class Lane, class SmsOf>
Lane* serve_admit(ServeQueue<Req>& s, std::vector<Lane>& lanes, SmsOf sms_of) {
    Lane* free_hi = nullptr;
    Lane* free_lo = nullptr;
    for (auto& L : lanes) {
        if (L.busy) continue;
        if (L.hi && !free_hi) free_hi = &L;
        if (!L.hi && !free_lo) free_lo = &L;
    }
    if (!free_hi && !free_lo) return nullptr;
    const size_t room = s.budget - std::min(s.budget, s.in_use);
    Req* big = s.large.empty() ? nullptr : s.large.front();
    Req* small = s.small.empty() ? nullptr : s.small.front();
    int P = 0;
    bool big_ok = false;
    if (big && free_lo) {
        P = sms_of(big->n);
        big_ok = (big->footprint <= room || s.in_use == 0) && (s.sms_used == 0 || s.sms_used + P <= s.sms_cap);
    }
    const bool small_ok = small && (small->footprint <= room || s.in_use == 0);
    if (small_ok && !(big_ok && big->bypassed >= SERVE_MAX_BYPASS)) {
        Lane& L = free_hi ? *free_hi : *free_lo;
        size_t used = 0;
        const auto pivot = small->pivot;
        const double tol = small->tol;
        for (auto it = s.small.begin(); it != s.small.end();) {
            Req* q = *it;
            if (q->pivot == pivot && q->tol == tol && (used + q->footprint <= room || L.reqs.empty()) &&
                L.reqs.size() < SERVE_MAX_BATCH) {
                used += q->footprint;
                L.reqs.push_back(q);
                it = s.small.erase(it);
            } else {
                ++it;
            }
        }
        if (big_ok) big->bypassed++;
        L.sms = 0;
        s.in_use += used;
        return &L;
    }
    if (!big_ok) return nullptr;
    Lane& L = *free_lo;
    s.large.pop_front();
    L.reqs.push_back(big);
    L.sms = P;
    s.sms_used += P;
    s.in_use += big->footprint;
    return &L;
}

// Gives back what a finished lane held; the caller clears its reqs.
template <class Req, class Lane>
void serve_release(ServeQueue<Req>& s, Lane& L) {
    for (Req* q : L.reqs) s.in_use -= q->footprint;
    s.sms_used -= L.sms;
    L.sms = 0;
}

}  // namespace pjac
