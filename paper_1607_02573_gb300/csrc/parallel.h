// A minimal host thread pool loop for the setup phase (partition, slot maps,
// symbolic analysis): parallel_for(n, fn) runs fn(i, worker) for i in [0, n)
// on up to hardware_concurrency threads with dynamic chunking.  Exceptions
// thrown by fn are rethrown on the calling thread.
#pragma once

#include <atomic>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace mwi {

inline int setup_threads() {
    unsigned h = std::thread::hardware_concurrency();
    return (int)(h == 0 ? 4 : (h > 64 ? 64 : h));
}

template <typename F>
void parallel_for(int64_t n, int64_t chunk, F&& fn) {
    const int nth = (int)std::min<int64_t>(setup_threads(), std::max<int64_t>(1, (n + chunk - 1) / chunk));
    if (nth <= 1) {
        for (int64_t i = 0; i < n; ++i) fn(i, 0);
        return;
    }
    std::atomic<int64_t> next{0};
    std::exception_ptr err;
    std::mutex mu;
    auto work = [&](int w) {
        try {
            for (;;) {
                const int64_t b = next.fetch_add(chunk);
                if (b >= n) break;
                const int64_t e = std::min(n, b + chunk);
                for (int64_t i = b; i < e; ++i) fn(i, w);
            }
        } catch (...) {
            std::lock_guard<std::mutex> lk(mu);
            if (!err) err = std::current_exception();
            next.store(n);
        }
    };
    std::vector<std::thread> th;
    for (int w = 1; w < nth; ++w) th.emplace_back(work, w);
    work(0);
    for (auto& t : th) t.join();
    if (err) std::rethrow_exception(err);
}

}  // namespace mwi
