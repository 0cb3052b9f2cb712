// Command-line driver of the batch autotuner's JSON store (no GPU):
//   tune_cache_cli <path> lookup <key>
//       prints "HIT key_bits radix_bits trace_block layout ms" or "MISS"
//   tune_cache_cli <path> store <key> <key_bits> <radix_bits> <trace_block> <layout> <ms>
//       prints "OK" or "FAIL <message>"
#include <cstdio>
#include <cstdlib>
#include <string>

#include "rr_tune_cache.h"

int main(int argc, char **argv) {
    if (argc < 4) return 2;
    const std::string path = argv[1], cmd = argv[2], key = argv[3];
    if (cmd == "lookup") {
        rr::TuneEntry e;
        if (rr::tune_cache_lookup(path, key, &e))
            std::printf("HIT %u %u %u %d %.6g\n", e.key_bits, e.radix_bits, e.trace_block, e.layout, e.ms);
        else
            std::printf("MISS\n");
        return 0;
    }
    if (cmd == "store" && argc == 9) {
        rr::TuneEntry e;
        e.key_bits = (uint32_t)std::strtoul(argv[4], nullptr, 10);
        e.radix_bits = (uint32_t)std::strtoul(argv[5], nullptr, 10);
        e.trace_block = (uint32_t)std::strtoul(argv[6], nullptr, 10);
        e.layout = (int32_t)std::strtol(argv[7], nullptr, 10);
        e.ms = std::strtod(argv[8], nullptr);
        std::string err;
        if (rr::tune_cache_store(path, key, e, &err))
            std::printf("OK\n");
        else
            std::printf("FAIL %s\n", err.c_str());
        return 0;
    }
    return 2;
}
