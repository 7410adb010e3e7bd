// launch_count.h -- running count of kernel launches issued by the library (host side).
#pragma once

#include <atomic>

namespace cng {

std::atomic<long long>& launch_counter();
inline void count_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

}  // namespace cng
