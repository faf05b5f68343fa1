"""Host model of ppf_execute_host's three-stage pipeline (csrc/ppf_api.cu).

Slices go through an upload stream, a kernel stream and a download stream and
three staging slots (slice s uses slot s mod 3).  Each stream runs its
operations in order; cudaStreamWaitEvent makes a stream wait for the event's
most recent record enqueued before the wait (a wait on a never-recorded event
is a no-op).  The enqueue order per slice is the library's: upload (after
waiting for the kernel of slice s - 3), record "in"; kernel (after "in" of s
and the download of slice s - 3), record "k"; download (after "k"), record
"out".  Any progress order of the three streams must upload, transform and
download every slice from slots that hold it; leaving out either reuse wait
lets a later slice overwrite a slot still in use.  Host-only: no GPU.
"""
import random

import pytest

SLOTS = 3


def enqueue(n_slices, drop_upload_wait=False, drop_kernel_wait=False):
    streams = {"up": [], "k": [], "down": []}
    last_record = {}  # event name -> id of its latest record op
    ops = {}

    def add(stream, kind, slice_, waits=()):
        oid = len(ops)
        deps = [last_record[e] for e in waits if e in last_record]
        ops[oid] = {"stream": stream, "kind": kind, "slice": slice_, "deps": deps}
        streams[stream].append(oid)
        return oid

    for s in range(n_slices):
        k = s % SLOTS
        reuse = s >= SLOTS
        up_waits = [f"k{k}"] if reuse and not drop_upload_wait else []
        add("up", "upload", s, up_waits)
        last_record[f"in{k}"] = add("up", "record", s)
        k_waits = [f"in{k}"] + ([f"out{k}"] if reuse and not drop_kernel_wait else [])
        add("k", "kernel", s, k_waits)
        last_record[f"k{k}"] = add("k", "record", s)
        add("down", "download", s, [f"k{k}"])
        last_record[f"out{k}"] = add("down", "record", s)
    return streams, ops


def run(n_slices, seed, **mistake):
    rng = random.Random(seed)
    streams, ops = enqueue(n_slices, **mistake)
    done = set()
    pos = {name: 0 for name in streams}
    slot_in = [None] * SLOTS
    slot_out = [None] * SLOTS
    downloaded = []
    while any(pos[n] < len(streams[n]) for n in streams):
        ready = [n for n in streams if pos[n] < len(streams[n])
                 and all(d in done for d in ops[streams[n][pos[n]]]["deps"])]
        assert ready, "pipeline deadlock"
        name = rng.choice(ready)
        oid = streams[name][pos[name]]
        op = ops[oid]
        k = op["slice"] % SLOTS
        if op["kind"] == "upload":
            slot_in[k] = op["slice"]
        elif op["kind"] == "kernel":
            assert slot_in[k] == op["slice"], f"slice {op['slice']} transformed from a slot holding {slot_in[k]}"
            slot_out[k] = op["slice"]
        elif op["kind"] == "download":
            assert slot_out[k] == op["slice"], f"slice {op['slice']} downloaded from a slot holding {slot_out[k]}"
            downloaded.append(op["slice"])
        done.add(oid)
        pos[name] += 1
    assert sorted(downloaded) == list(range(n_slices))


@pytest.mark.parametrize("n_slices", [1, 2, 3, 4, 7, 25])
def test_pipeline_moves_every_slice_through_its_own_slots(n_slices):
    for seed in range(200):
        run(n_slices, seed)


@pytest.mark.parametrize("mistake", ["drop_upload_wait", "drop_kernel_wait"])
def test_pipeline_without_a_reuse_wait_fails(mistake):
    with pytest.raises(AssertionError, match="from a slot holding"):
        for seed in range(200):
            run(7, seed, **{mistake: True})
