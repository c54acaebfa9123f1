// Launch accounting and optional per-kernel CUDA-event timing, shared by the
// single-solve handle and the batch handle.  While enabled, each enqueued
// kernel is bracketed by event-record nodes (cudaEventRecordExternal) so the
// timing survives graph capture; collect() adds each bracket's device time to
// a record keyed by (kernel name, level) after a graph run.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "gmg.h"

namespace gmg {

struct KernelTimer {
    bool enabled = false;
    int graph_kernels = 0;  // kernel launches per graph run
    int64_t launches = 0;   // launches since the last reset
    struct Pending {
        std::string name;
        int level;
        double ops, bytes;
        int group;  // cur_group at enqueue time
    };
    // Launches enqueued while cur_group = g > 0 belong to group g; a graph run
    // whose device-side plan skipped group g passes bit g to after_graph_run,
    // which then leaves their (empty) brackets out of the records.
    int cur_group = 0;
    std::vector<Pending> pending;  // timed launches of one graph, in order
    std::vector<cudaEvent_t> ev;   // two per timed launch
    struct Stat {
        int64_t launches = 0;
        double ms = 0.0, ops = 0.0, bytes = 0.0;
    };
    std::map<std::pair<std::string, int>, Stat> stats;

    void begin_capture() {
        pending.clear();
        graph_kernels = 0;
    }

    // launch() enqueues `kernels` kernels on s.
    template <class F>
    void run(cudaStream_t s, const std::string& name, int level, double ops, double bytes,
             int kernels, F&& launch) {
        if (enabled) {
            const size_t i = pending.size();
            while (ev.size() < 2 * (i + 1)) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ev.push_back(e);
            }
            cudaEventRecordWithFlags(ev[2 * i], s, cudaEventRecordExternal);
            launch();
            cudaEventRecordWithFlags(ev[2 * i + 1], s, cudaEventRecordExternal);
            pending.push_back({name, level, ops, bytes, cur_group});
        } else {
            launch();
        }
        graph_kernels += kernels;
    }

    // After a run of the captured graph.
    void after_graph_run(unsigned skipped_groups = 0) {
        launches += graph_kernels;
        if (!enabled) return;
        for (size_t i = 0; i < pending.size(); ++i) {
            if (pending[i].group > 0 && (skipped_groups >> pending[i].group & 1u)) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            auto& p = pending[i];
            auto& st = stats[{p.name, p.level}];
            st.launches++;
            st.ms += ms;
            st.ops = p.ops;
            st.bytes = p.bytes;
        }
    }

    void reset() {
        stats.clear();
        launches = 0;
    }

    void destroy() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
    }

    void report(gmg_kernel_stat* out, int cap, int* count, int64_t* launches_out) const {
        int i = 0;
        for (auto& kv : stats) {
            if (i < cap) {
                gmg_kernel_stat& s = out[i];
                std::memset(&s, 0, sizeof(s));
                std::snprintf(s.kernel, sizeof(s.kernel), "%s", kv.first.first.c_str());
                s.level = kv.first.second;
                s.launches = kv.second.launches;
                s.ms = kv.second.ms;
                s.dp_ops = kv.second.ops;
                s.bytes = kv.second.bytes;
            }
            ++i;
        }
        if (count) *count = i;
        if (launches_out) *launches_out = launches;
    }
};

}  // namespace gmg
