// Run order of a packed batch (kgpu::hostutil::order_batch), on the CPU.
// Reads "reserve n" then n lines "mode nblocks unit_blocks tile_units refused"
// from stdin; prints the run order, then the tile prefix (n + 1 values).
#include <cstdio>
#include <vector>

#include "kgpu_ctx.h"

int main() {
    unsigned long long reserve = 0;
    unsigned n = 0;
    if (std::scanf("%llu %u", &reserve, &n) != 2) return 2;
    std::vector<kgpu::ReqDesc> d(n);
    std::vector<int> refused(n);
    for (unsigned i = 0; i < n; i++) {
        unsigned mode, ub, tu;
        unsigned long long nb;
        if (std::scanf("%u %llu %u %u %d", &mode, &nb, &ub, &tu, &refused[i]) != 5) return 2;
        d[i] = kgpu::ReqDesc{};
        d[i].mode = mode;
        d[i].nblocks = nb;
        d[i].unit_blocks = ub;
        d[i].tile_units = tu;
    }
    std::vector<uint64_t> prefix(n + 1);
    std::vector<uint32_t> order(n);
    kgpu::hostutil::order_batch(d.data(), n, [&](uint32_t i) { return refused[i] != 0; }, reserve, prefix.data(),
                                order.data());
    for (unsigned i = 0; i < n; i++) std::printf("%u ", order[i]);
    std::printf("\n");
    for (unsigned i = 0; i <= n; i++) std::printf("%llu ", (unsigned long long)prefix[i]);
    std::printf("\n");
    return 0;
}
