// Per-call argument checks of the XTS entry points (kgpu::hostutil::xts_args)
// and the registered-host-range lookup (kgpu::hostutil::host_translate), on
// the CPU, against a fake context whose registered ranges are
//   [0x1000, 0x2000) seen by the device at +0x100000,
//   [0x2000, 0x3000) at +0x200000 (adjacent to the first),
//   [0x5000, 0x9000) at +0x300000,
//   [0x10000, 0x11000) at +0 (mapped at the same address).
// Reads lines
//   "x dir len du sector stealing"  -> prints the return code of xts_args
//   "h p len"                        -> prints the return code and the device address
// (numbers in decimal, p in hex).
#include <cstdio>

#include "kgpu_ctx.h"

int main() {
    kgpu_ctx* ctx = new kgpu_ctx();
    const unsigned long long ranges[4][3] = {
        {0x1000, 0x2000, 0x100000}, {0x2000, 0x3000, 0x200000}, {0x5000, 0x9000, 0x300000}, {0x10000, 0x11000, 0}};
    for (const auto& r : ranges) {
        kgpu::HostRange h;
        h.base = (uintptr_t)r[0];
        h.end = (uintptr_t)r[1];
        h.dev_off = (intptr_t)r[2];
        ctx->hreg.push_back(h);
    }
    char kind[2];
    while (std::scanf("%1s", kind) == 1) {
        if (kind[0] == 'x') {
            int dir, stealing;
            unsigned long long len, du, sector;
            if (std::scanf("%d %llu %llu %llu %d", &dir, &len, &du, &sector, &stealing) != 5) return 2;
            std::printf("%d\n", kgpu::hostutil::xts_args(ctx, dir, (size_t)len, (size_t)du, sector, stealing != 0));
        } else if (kind[0] == 'h') {
            unsigned long long p, len;
            if (std::scanf("%llx %llu", &p, &len) != 2) return 2;
            uintptr_t dev = 0;
            const int r = kgpu::hostutil::host_translate(ctx, reinterpret_cast<const void*>((uintptr_t)p), (size_t)len,
                                                         &dev);
            std::printf("%d %llx\n", r, (unsigned long long)dev);
        } else {
            return 2;
        }
    }
    delete ctx;
    return 0;
}
