"""The seeded input generators (CPU): SplitMix64 against its published first outputs and a
plain-integer restatement, and the properties the workload recipes rely on (tamper plans,
length and size ranges, counter-mode BPV subsets, key material ranges)."""
import numpy as np

from paper_2506_08781_gb300 import synth

M64 = (1 << 64) - 1


def _mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_published_outputs_and_plain_restatement():
    # SplitMix64 from state 0: the first two outputs of the reference generator
    first = synth._mix64(np.array([0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) & M64], dtype=np.uint64))
    assert [int(x) for x in first] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    for seed, tag in [(0, "msg"), (7, "tamper.idx"), (2 ** 63 + 5, "key")]:
        s = int(synth._stream_seed(seed, tag))
        want = [_mix((s + k * 0x9E3779B97F4A7C15) & M64) for k in range(11, 11 + 40)]
        assert [int(x) for x in synth.words(seed, tag, 40, start=10)] == want


def test_tamper_plan_properties():
    msgs = synth.messages(5, 500, 1, 300)
    plan = synth.tamper_plan(5, msgs, 60)
    assert list(plan.idx) == sorted(set(plan.idx.tolist())) and len(plan.idx) == 60
    lens = (msgs.offs[1:] - msgs.offs[:-1]).astype(np.int64)
    assert np.all(plan.pos >= 0) and np.all(plan.pos < lens[plan.idx])
    assert np.all(plan.mask >= 1)
    bad = synth.apply_tamper(msgs, plan)
    diff = np.nonzero(bad.data != msgs.data)[0]
    assert list(diff) == sorted((msgs.offs[plan.idx].astype(np.int64) + plan.pos).tolist())
    assert np.array_equal(bad.offs, msgs.offs)


def test_ranges_of_lengths_sizes_and_keys():
    msgs = synth.messages(9, 4000, 32, 256)
    lens = (msgs.offs[1:] - msgs.offs[:-1]).astype(np.int64)
    assert lens.min() >= 32 and lens.max() <= 256 and 120 < lens.mean() < 168
    sizes = synth.device_sizes(9, 4096, 16, 65536)
    assert sizes.min() >= 16 and sizes.max() <= 65536
    # log-uniform: the median sits near the geometric mean of the range (16 * 65537)^(1/2) ~ 1024
    assert 700 < np.median(sizes) < 1500
    for s in range(20):
        km = synth.key_material(s, v=8)
        y = int.from_bytes(km.y, "little")
        assert 0 < y < 2 ** 252
        assert all(int.from_bytes(km.bpv_r[32 * k:32 * k + 32].tobytes(), "little") < 2 ** 252 for k in range(8))


def test_bpv_subsets_are_counter_mode():
    """Entry t's subset depends only on (seed, t): signing a log in pieces gives the same
    subsets as signing it whole."""
    whole = synth.bpv_subsets(3, 40, v=64, k=4)
    assert whole.max() < 64
    assert np.array_equal(synth.bpv_subsets(3, 15, first_index=10, v=64, k=4), whole[10:25])
