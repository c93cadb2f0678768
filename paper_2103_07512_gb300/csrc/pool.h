// pool.h -- a small fixed pool of host worker threads for parallel loops of
// the compiler (planning the tree groups of a population concurrently).
//
// run(n, body) calls body(0..n-1), each index exactly once, on the pool's
// workers and on the calling thread, and returns when every call has
// returned.  Several threads may call run at the same time.  The pool never
// touches a batch after its caller has returned: a worker announces that it
// holds a batch (under the lock) before claiming indices from it, and the
// caller waits until no worker holds its batch.
#pragma once
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace tgp {

class WorkerPool {
public:
    explicit WorkerPool(int n_workers) {
        for (int i = 0; i < n_workers; ++i) threads_.emplace_back([this] { work(); });
    }
    ~WorkerPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        wake_.notify_all();
        for (auto& t : threads_) t.join();
    }
    WorkerPool(const WorkerPool&) = delete;
    WorkerPool& operator=(const WorkerPool&) = delete;

    int workers() const { return (int)threads_.size(); }

    void run(int n, const std::function<void(int)>& body) {
        if (n <= 0) return;
        if (n == 1 || threads_.empty()) {
            for (int i = 0; i < n; ++i) body(i);
            return;
        }
        Batch b;
        b.body = &body;
        b.n = n;
        {
            std::lock_guard<std::mutex> g(mu_);
            queue_.push_back(&b);
        }
        wake_.notify_all();
        drain(&b);
        std::unique_lock<std::mutex> lk(mu_);
        auto it = std::find(queue_.begin(), queue_.end(), &b);
        if (it != queue_.end()) queue_.erase(it);
        done_.wait(lk, [&] { return b.holders == 0 && b.finished.load() == n; });
    }

private:
    struct Batch {
        const std::function<void(int)>* body = nullptr;
        int n = 0;
        std::atomic<int> next{0};
        std::atomic<int> finished{0};
        int holders = 0;   // workers inside drain(), guarded by mu_
    };

    std::mutex mu_;
    std::condition_variable wake_, done_;
    std::deque<Batch*> queue_;
    std::vector<std::thread> threads_;
    bool stop_ = false;

    // Claims and runs indices of b until none is left.
    static void drain(Batch* b) {
        for (;;) {
            const int i = b->next.fetch_add(1);
            if (i >= b->n) return;
            (*b->body)(i);
            b->finished.fetch_add(1);
        }
    }

    void work() {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            wake_.wait(lk, [&] { return stop_ || !queue_.empty(); });
            if (stop_) return;
            Batch* b = queue_.front();
            if (b->next.load() >= b->n) {   // nothing left to claim: retire it from the queue
                queue_.pop_front();
                continue;
            }
            ++b->holders;
            lk.unlock();
            drain(b);
            lk.lock();
            --b->holders;
            if (b->holders == 0) done_.notify_all();
        }
    }
};

}  // namespace tgp
