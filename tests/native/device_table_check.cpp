// Host-only check of the per-device kernel-attribute record
// (paper_2301_09349_gb300/csrc/device_table.h): a limit applied on one device
// does not count for another, a larger request is applied again, a failed
// application is not recorded, and concurrent host threads apply each
// (kernel, device) limit once.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "device_table.h"

static int kernel_a, kernel_b;   // stand-ins for two kernels' addresses

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            std::printf("FAILED %s (line %d)\n", #c, __LINE__);   \
            return 1;                                             \
        }                                                         \
    } while (0)

int main() {
    ibmk::DeviceAttrTable t;
    int applied = 0;
    auto ok = [&]() { ++applied; return 0; };
    CHECK(t.ensure(&kernel_a, 0, 70000, ok) == 0 && applied == 1);
    CHECK(t.ensure(&kernel_a, 0, 70000, ok) == 0 && applied == 1);   // recorded
    CHECK(t.ensure(&kernel_a, 0, 60000, ok) == 0 && applied == 1);   // smaller: covered
    CHECK(t.ensure(&kernel_a, 1, 70000, ok) == 0 && applied == 2);   // other device
    CHECK(t.ensure(&kernel_b, 0, 70000, ok) == 0 && applied == 3);   // other kernel
    CHECK(t.ensure(&kernel_a, 0, 90000, ok) == 0 && applied == 4);   // larger: again
    CHECK(t.recorded(&kernel_a, 0) == 90000 && t.recorded(&kernel_a, 1) == 70000);
    CHECK(t.recorded(&kernel_b, 1) == 0);
    // a failing application returns its code and records nothing
    CHECK(t.ensure(&kernel_b, 1, 80000, []() { return 98; }) == 98);
    CHECK(t.recorded(&kernel_b, 1) == 0);
    CHECK(t.ensure(&kernel_b, 1, 80000, ok) == 0 && applied == 5);
    // eight threads on four devices: one application per device
    ibmk::DeviceAttrTable t2;
    std::atomic<int> count{0};
    std::vector<std::thread> th;
    for (int i = 0; i < 8; ++i)
        th.emplace_back([&, i]() {
            for (int r = 0; r < 1000; ++r)
                t2.ensure(&kernel_a, i % 4, 100000, [&]() { count.fetch_add(1); return 0; });
        });
    for (auto &x : th) x.join();
    CHECK(count.load() == 4);
    std::printf("device table ok\n");
    return 0;
}
