// Request validation of batched and served requests (kgpu::hostutil::make_desc),
// on the CPU, against a fake context:
//   key handles 1 (XTS, live), 2 (single key, live), 3 (XTS, deleted);
//   device allocations [0x10000000, +1 MiB) and [0x20000000, +1 MiB), seen
//   through a stand-in for the range cache (no CUDA call is made);
//   one registered host range [0x70000000, +1 MiB), mapped for the device at
//   +0x1000000000.
// Reads "tile_chunks" then lines "mode dir key flags src dst len unit sector ivs"
// (addresses in hex); prints per line the return code and the descriptor:
// "rc src dst ivs nblocks first_sector unit_blocks key mode dir flags tile_units".
#include <cstdio>
#include <utility>
#include <vector>

#include "kgpu_ctx.h"

namespace {

struct FakeAllocations {
    std::vector<std::pair<uintptr_t, uintptr_t>> r{{0x10000000u, 0x10000000u + (1u << 20)},
                                                  {0x20000000u, 0x20000000u + (1u << 20)}};
    int check(const kgpu_ctx*, const void* p, size_t len) const {
        const uintptr_t a = (uintptr_t)p, e = a + len;
        if (!p || e < a) return KGPU_EFAULT;
        for (const auto& x : r)
            if (a >= x.first && a < x.second) return e <= x.second ? KGPU_OK : KGPU_EFAULT;
        return KGPU_EFAULT;
    }
};

}  // namespace

int main() {
    kgpu_ctx* ctx = new kgpu_ctx();
    ctx->keys.resize(3);
    ctx->keys[0].live = true;
    ctx->keys[0].xts = true;
    ctx->keys[1].live = true;
    ctx->keys[1].xts = false;
    ctx->keys[2].live = false;
    ctx->keys[2].xts = true;
    kgpu::HostRange h;
    h.base = 0x70000000u;
    h.end = h.base + (1u << 20);
    h.dev_off = (intptr_t)0x1000000000ll;
    ctx->hreg.push_back(h);

    unsigned tile_chunks = 0;
    if (std::scanf("%u", &tile_chunks) != 1) return 2;
    unsigned mode, dir, key, flags;
    unsigned long long src, dst, len, unit, sector, ivs;
    while (std::scanf("%u %u %u %u %llx %llx %llu %llu %llu %llx", &mode, &dir, &key, &flags, &src, &dst, &len, &unit,
                      &sector, &ivs) == 10) {
        kgpu_request q{};
        q.mode = mode;
        q.dir = dir;
        q.key = key;
        q.flags = flags;
        q.src = reinterpret_cast<const void*>((uintptr_t)src);
        q.dst = reinterpret_cast<void*>((uintptr_t)dst);
        q.len = len;
        q.unit_size = unit;
        q.sector = sector;
        q.ivs = reinterpret_cast<const uint8_t*>((uintptr_t)ivs);
        FakeAllocations rc;
        kgpu::ReqDesc d{};
        const int r = kgpu::hostutil::make_desc(ctx, q, rc, tile_chunks, &d);
        std::printf("%d %llx %llx %llx %llu %llu %u %u %u %u %u %u\n", r, (unsigned long long)(uintptr_t)d.src,
                    (unsigned long long)(uintptr_t)d.dst, (unsigned long long)(uintptr_t)d.ivs,
                    (unsigned long long)d.nblocks, (unsigned long long)d.first_sector, d.unit_blocks, d.key, d.mode,
                    d.dir, d.flags, d.tile_units);
    }
    delete ctx;
    return 0;
}
