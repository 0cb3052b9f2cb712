// Host-side store of the batch autotuner's choices: one JSON file mapping a
// key (GPU, batch-size bucket, key layout and estimate, wavefront bits) to
// the configuration the tuner picked and its time.
#pragma once

#include <stdint.h>

#include <string>

namespace rr {

struct TuneEntry {
    uint32_t key_bits = 0;
    uint32_t radix_bits = 0;
    uint32_t trace_block = 0;
    int32_t layout = -1;
    double ms = 0.0;
};

// The file's format:
//   {"format": "rr-batch-tune-cache", "version": 1,
//    "entries": {"<key>": {"key_bits": 24, "radix_bits": 8, "trace_block": 128,
//                          "layout": -1, "ms": 8.12}, ...}}
// A missing, unreadable or malformed file holds no entries.

// True and *e filled when `path` holds an entry for `key`.
bool tune_cache_lookup(const std::string &path, const std::string &key, TuneEntry *e);

// Adds or replaces the entry for `key`, keeping the file's other entries.
// The file is written to a temporary name in the same directory and renamed
// over `path`, so a reader never sees a partly written file.  False (with a
// message) when the file cannot be written.
bool tune_cache_store(const std::string &path, const std::string &key, const TuneEntry &e, std::string *err);

}  // namespace rr
