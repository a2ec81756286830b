// Process-wide worker pool behind parallel_for (host sift, staging copies):
// threads are started once instead of per loop, which matters for loops of
// a millisecond or less run several times per file.
#include <condition_variable>
#include <deque>
#include <mutex>

#include "pss_internal.h"

namespace pss {

namespace {

struct Job {
    const std::function<void(int64_t)>* f;
    int64_t n, grain;
    std::atomic<int64_t> next{0};
    int entries = 0;   // queue entries posted for workers
    int finished = 0;  // entries taken and completed (under the pool lock)
};

class Pool {
  public:
    Pool() {
        const unsigned hc = std::thread::hardware_concurrency();
        const int k = hc > 1 ? (int)std::min(hc - 1, 63u) : 0;
        for (int i = 0; i < k; ++i) th_.emplace_back([this] { run(); });
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    int workers() const { return (int)th_.size(); }

    void run_job(Job* j) {
        const int64_t chunks = (j->n + j->grain - 1) / j->grain;
        const int want = (int)std::min<int64_t>(workers(), chunks - 1);
        {
            std::lock_guard<std::mutex> lk(mu_);
            j->entries = want;
            for (int i = 0; i < want; ++i) q_.push_back(j);
        }
        if (want > 0) cv_.notify_all();
        work(j);
        std::unique_lock<std::mutex> lk(mu_);
        // entries no worker has taken yet are withdrawn; wait for the ones taken
        for (auto it = q_.begin(); it != q_.end();)
            if (*it == j) {
                it = q_.erase(it);
                ++j->finished;
            } else {
                ++it;
            }
        done_.wait(lk, [&] { return j->finished == j->entries; });
    }

  private:
    static void work(Job* j) {
        for (;;) {
            const int64_t b = j->next.fetch_add(j->grain);
            if (b >= j->n) return;
            const int64_t e = std::min(j->n, b + j->grain);
            for (int64_t i = b; i < e; ++i) (*j->f)(i);
        }
    }
    void run() {
        for (;;) {
            Job* j = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
                if (stop_) return;
                j = q_.front();
                q_.pop_front();
            }
            work(j);
            {
                std::lock_guard<std::mutex> lk(mu_);
                ++j->finished;
            }
            done_.notify_all();
        }
    }

    std::mutex mu_;
    std::condition_variable cv_, done_;
    std::deque<Job*> q_;
    std::vector<std::thread> th_;
    bool stop_ = false;
};

Pool& pool() {
    static Pool p;
    return p;
}

}  // namespace

void parallel_for_fn(int64_t n, int64_t grain, const std::function<void(int64_t)>& f) {
    if (grain < 1) grain = 1;
    Job j;
    j.f = &f;
    j.n = n;
    j.grain = grain;
    pool().run_job(&j);
}

}  // namespace pss
