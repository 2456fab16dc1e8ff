// dfr_tickets.h -- host-only pieces of the served form that need no CUDA:
// the ticket table's poll / wait and the start of the dispatcher thread.
// Kept free of CUDA so that the CPU tests can compile them on their own and
// drive them with several threads.
#pragma once

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>

namespace dfr {

// Result of looking a ticket up.
enum class Ticket { unknown, pending, done };

// With the table's mutex held: if `ticket` is done, remove it from the table
// and hand its request to the caller (who deletes it); R must have a `done`
// flag.
template <class R>
Ticket take_if_done(std::unordered_map<uint64_t, R*>& table, uint64_t ticket, R** out) {
  *out = nullptr;
  auto it = table.find(ticket);
  if (it == table.end()) return Ticket::unknown;
  if (!it->second->done) return Ticket::pending;
  *out = it->second;
  table.erase(it);
  return Ticket::done;
}

// Block (mutex held through `lk`, released while waiting on `cv`) until
// `ticket` is done, then take it as take_if_done does.  The ticket is looked
// up again after every wait: another thread polling or waiting on the same
// ticket may take (and free) the request meanwhile, and then this call
// returns Ticket::unknown without touching it.
template <class R>
Ticket wait_and_take(std::unique_lock<std::mutex>& lk, std::condition_variable& cv,
                     std::unordered_map<uint64_t, R*>& table, uint64_t ticket, R** out) {
  for (;;) {
    const Ticket t = take_if_done(table, ticket, out);
    if (t != Ticket::pending) return t;
    cv.wait_for(lk, std::chrono::milliseconds(1));
  }
}

// Start `fn` on a new thread made by `spawn(fn)` (normally std::thread's
// constructor).  Returns false, with *out untouched, when the system refuses
// the thread (std::system_error) or memory runs out: no exception crosses the
// C boundary above.
template <class F, class Spawn>
bool start_thread(std::thread* out, F&& fn, Spawn&& spawn) noexcept {
  try {
    *out = spawn(std::forward<F>(fn));
    return true;
  } catch (...) {
    return false;
  }
}

struct SpawnStdThread {
  template <class F>
  std::thread operator()(F&& fn) const {
    return std::thread(std::forward<F>(fn));
  }
};

}  // namespace dfr
