// host_parts.h -- host-side helpers of the library that need no CUDA: an
// allocator that leaves new elements unset, and run_parts, which splits host
// work over a persistent set of worker threads.
#pragma once

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <exception>
#include <memory>
#include <mutex>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

namespace rsv {

// An allocator whose value-less construct leaves the element default-initialised
// (no zero fill of large trivially copyable arrays that are written next).
template <class T>
struct DefaultInit : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = DefaultInit<U>;
    };
    using std::allocator<T>::allocator;
    template <class U>
    void construct(U* p) noexcept {
        ::new (static_cast<void*>(p)) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
    }
};

// Host worker threads kept for run_parts: starting a thread costs tens of
// microseconds, so a call that splits its work sixteen ways several times
// would spend milliseconds starting threads.  Parts are claimed from one
// counter tagged with the job's number, so a worker that wakes late can never
// take a part of a later job; the caller claims parts too, so a job finishes
// even with no worker (none started, or none left after a fork).  One job at
// a time: a concurrent caller starts its own threads.
class PartPool {
  public:
    static PartPool& get() {
        static PartPool pool;
        return pool;
    }
    // fn(ctx, k) for k = 0 .. T-1; false (nothing run) if the pool is busy or
    // the call comes from inside one of its parts
    bool run(int T, void (*fn)(void*, int), void* ctx) {
        if (in_part()) return false;
        std::unique_lock<std::mutex> use(use_, std::try_to_lock);
        if (!use.owns_lock()) return false;
        start_workers(T - 1);
        uint32_t g;
        {
            std::lock_guard<std::mutex> l(m_);
            g = ++gen_;
            fn_ = fn;
            ctx_ = ctx;
            T_ = T;
            done_ = 0;
            next_.store((uint64_t)g << 32);
        }
        cv_.notify_all();
        std::exception_ptr err;
        in_part() = true;
        for (int k; (k = claim(g, T)) >= 0;) {
            try {
                fn(ctx, k);
            } catch (...) {   // the other parts still run; the first error is rethrown
                if (!err) err = std::current_exception();
            }
            count(g);
        }
        in_part() = false;
        {
            std::unique_lock<std::mutex> l(m_);
            done_cv_.wait(l, [&] { return done_ == T; });
        }
        if (err) std::rethrow_exception(err);
        return true;
    }
    ~PartPool() {
        {
            std::lock_guard<std::mutex> l(m_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : workers_) t.join();
    }

  private:
    static bool& in_part() {   // this thread is running a part
        static thread_local bool f = false;
        return f;
    }
    int claim(uint32_t g, int T) {
        uint64_t v = next_.load();
        for (;;) {
            if ((uint32_t)(v >> 32) != g || (int)(uint32_t)v >= T) return -1;
            if (next_.compare_exchange_weak(v, v + 1)) return (int)(uint32_t)v;
        }
    }
    void count(uint32_t g) {
        std::lock_guard<std::mutex> l(m_);
        if (g == gen_ && ++done_ == T_) done_cv_.notify_all();
    }
    void start_workers(int want) {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        want = std::min(want, std::min(hw - 1, 15));
        try {
            while ((int)workers_.size() < want) workers_.emplace_back([this] { loop(); });
        } catch (...) {   // fewer workers: the caller claims the rest
        }
    }
    void loop() {
        in_part() = true;
        uint32_t seen = 0;
        for (;;) {
            void (*fn)(void*, int);
            void* ctx;
            int T;
            uint32_t g;
            {
                std::unique_lock<std::mutex> l(m_);
                cv_.wait(l, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = g = gen_;
                fn = fn_;
                ctx = ctx_;
                T = T_;
            }
            for (int k; (k = claim(g, T)) >= 0;) {
                fn(ctx, k);
                count(g);
            }
        }
    }
    std::mutex use_, m_;
    std::condition_variable cv_, done_cv_;
    std::vector<std::thread> workers_;
    std::atomic<uint64_t> next_{0};
    void (*fn_)(void*, int) = nullptr;
    void* ctx_ = nullptr;
    int T_ = 0, done_ = 0;
    uint32_t gen_ = 0;
    bool stop_ = false;
};

// Run part(k) for k = 0 .. T-1 on the pool's workers and this thread (or, if
// the pool is busy, on T - 1 helper threads and this one; parts whose thread
// cannot start run here).
template <class F>
inline void run_parts(int T, F&& part) {
    if (T <= 1) {
        if (T == 1) part(0);
        return;
    }
    using P = typename std::remove_reference<F>::type;
    if (PartPool::get().run(T, [](void* c, int k) { (*static_cast<P*>(c))(k); },
                            const_cast<void*>(static_cast<const void*>(&part))))
        return;
    std::vector<std::thread> th;
    int started = 1;
    try {
        th.reserve(T - 1);
        for (int k = 1; k < T; ++k) {
            th.emplace_back(part, k);
            ++started;
        }
    } catch (...) {   // no more threads: the rest runs serially below
    }
    part(0);
    for (int k = started; k < T; ++k) part(k);
    for (auto& t : th) t.join();
}

}  // namespace rsv
