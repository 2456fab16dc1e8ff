// CPU check of the served form's host-only pieces (dfr_tickets.h), built and
// run by tests/test_server_host.py under AddressSanitizer:
//   tickets  -- several threads wait on or poll one ticket while another
//               thread completes it: exactly one consumer takes the request,
//               every other one is told the ticket is gone, and no thread
//               touches the request after it was freed;
//   refused  -- a thread start that the system refuses is reported as a
//               failure instead of an exception.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <system_error>
#include <vector>

#include "dfr_tickets.h"

namespace {

struct Req {
  bool done = false;
  int status = 0;
};

int check_tickets(int waiters, int pollers, int rounds) {
  for (int round = 0; round < rounds; ++round) {
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, Req*> table;
    const uint64_t ticket = 7 + (uint64_t)round;
    Req* r = new Req();
    r->status = 40 + round;
    table[ticket] = r;
    std::atomic<int> took{0}, gone{0}, wrong{0};
    std::vector<std::thread> ts;
    for (int i = 0; i < waiters; ++i)
      ts.emplace_back([&] {
        std::unique_lock<std::mutex> lk(mu);
        Req* got = nullptr;
        const dfr::Ticket t = dfr::wait_and_take(lk, cv, table, ticket, &got);
        if (t == dfr::Ticket::done) {
          if (got->status != 40 + round) ++wrong;
          delete got;
          ++took;
        } else if (t == dfr::Ticket::unknown) {
          ++gone;
        } else {
          ++wrong;
        }
      });
    for (int i = 0; i < pollers; ++i)
      ts.emplace_back([&] {
        for (;;) {
          std::unique_lock<std::mutex> lk(mu);
          Req* got = nullptr;
          const dfr::Ticket t = dfr::take_if_done(table, ticket, &got);
          if (t == dfr::Ticket::pending) {
            lk.unlock();
            std::this_thread::yield();
            continue;
          }
          if (t == dfr::Ticket::done) {
            if (got->status != 40 + round) ++wrong;
            delete got;
            ++took;
          } else {
            ++gone;
          }
          return;
        }
      });
    std::this_thread::sleep_for(std::chrono::milliseconds(2));
    {
      std::lock_guard<std::mutex> lk(mu);
      r->done = true;  // the completion path marks it done under the mutex
    }
    cv.notify_all();
    for (auto& t : ts) t.join();
    if (took != 1 || gone != waiters + pollers - 1 || wrong != 0 || !table.empty()) {
      std::printf("tickets: round %d took=%d gone=%d wrong=%d left=%zu\n", round, took.load(), gone.load(),
                  wrong.load(), table.size());
      return 1;
    }
  }
  std::printf("tickets ok\n");
  return 0;
}

struct RefuseSpawn {
  template <class F>
  std::thread operator()(F&&) const {
    throw std::system_error(std::make_error_code(std::errc::resource_unavailable_try_again));
  }
};

int check_refused() {
  std::thread t;
  bool ran = false;
  const bool ok = dfr::start_thread(&t, [&ran] { ran = true; }, RefuseSpawn{});
  if (ok || t.joinable() || ran) {
    std::printf("refused: start_thread reported %d\n", (int)ok);
    return 1;
  }
  std::atomic<bool> ran2{false};
  if (!dfr::start_thread(&t, [&ran2] { ran2 = true; }, dfr::SpawnStdThread{}) || !t.joinable()) {
    std::printf("refused: a normal start failed\n");
    return 1;
  }
  t.join();
  if (!ran2) return 1;
  std::printf("refused ok\n");
  return 0;
}

}  // namespace

int main(int argc, char** argv) {
  const char* what = argc > 1 ? argv[1] : "all";
  int rc = 0;
  if (!std::strcmp(what, "tickets") || !std::strcmp(what, "all")) rc |= check_tickets(3, 2, 200);
  if (!std::strcmp(what, "refused") || !std::strcmp(what, "all")) rc |= check_refused();
  return rc;
}
