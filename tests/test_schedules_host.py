"""The execute-schedule enumeration (host logic, no GPU needed): for every FFT length the
library can convert, the default schedule comes first and every schedule is a valid split of
the transform that the kernels' static shape rules accept."""
import pytest

FP64, FP32 = 0, 1
SMEM_MAX = 232448  # bytes of dynamic shared memory a CTA may opt into


@pytest.fixture(scope="module")
def tdh():
    from paper_1604_07486_gb300 import build
    import paper_1604_07486_gb300 as m
    build.build()
    return m


def _radix(prec, logLC):
    return 16 if prec == FP32 and logLC > 9 else 8


def _passes(logLC, R):
    """Radices of the local passes: radix-R passes and a trailing smaller radix."""
    logR = R.bit_length() - 1
    npr = logLC // logR
    rest = 1 << (logLC - npr * logR)
    return [R] * npr + ([rest] if rest > 1 else [])


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_default_schedule_rule(tdh, prec):
    """Default: the largest local FFT shared memory holds (2^14 float32, 2^13 float64), the
    fewest CTAs per vector; half-size slices for multi-pass FFTs of up to 128 full slices."""
    cap = 14 if prec == FP32 else 13
    for logL in range(8, cap + 10):  # up to 512 slices
        sched = tdh.compiled_schedules(prec, logL)
        d = sched[0]
        if logL <= cap:
            assert (d["logLC"], d["C"]) == (logL, 1), (logL, d)
        elif (1 << (logL - cap)) <= 8:
            assert (d["logLC"], d["C"]) == (cap, 1 << (logL - cap)), (logL, d)
        elif (1 << (logL - cap)) <= 128:
            assert (d["logLC"], d["C"], d["multipass"]) == (cap - 1, 1 << (logL - cap + 1), 1)
            assert any(s["multipass"] == 2 for s in sched)  # the TMA variant is a candidate
        else:
            assert (d["logLC"], d["C"], d["multipass"]) == (cap, 1 << (logL - cap), 1)
        assert d["MINB"] == (2 if d["multipass"] and d["logLC"] == cap - 1 else 1)
        if d["multipass"]:  # float32 multi-pass slices default to radix 32
            assert d["R"] == (32 if prec == FP32 else 8), d


@pytest.mark.parametrize("ragged", [False, True])
@pytest.mark.parametrize("prec", [FP32, FP64])
def test_every_schedule_is_a_valid_split(tdh, prec, ragged):
    seen_any = 0
    for logL in range(8, (14 if prec == FP32 else 13) + 10):
        sched = tdh.compiled_schedules(prec, logL, ragged)
        keys = [(s["logLC"], s["C"], s["NT"], s["MINB"], s["multipass"], s["R"]) for s in sched]
        assert len(set(keys)) == len(keys), (logL, keys)
        for s in sched:
            seen_any += 1
            lc, C, R, NT = s["logLC"], s["C"], s["R"], s["NT"]
            assert lc + C.bit_length() - 1 == logL, (logL, s)
            if R == 32:
                # radix-32 passes, float32 only: 2^14-point slices on 512 threads, one CTA or
                # 2-8-CTA clusters, and single-CTA 2^13-point FFTs on 256 threads, two CTAs per
                # SM (their accumulators live in tensor memory); the multi-pass kernels' slices
                # (plain cross stage)
                assert prec == FP32, s
                assert (lc == 14 and C <= 8 and NT == 512 and s["MINB"] == 1) or \
                    (lc == 13 and C == 1 and NT == 256 and s["MINB"] == 2) or \
                    (C > 8 and s["multipass"] == 1), s
            else:
                assert R == _radix(prec, lc)
            if C > 8:
                # 2: the cross stage moves its blocks with bulk tensor copies (16 ... 256 slices)
                assert s["multipass"] in ((1, 2) if C <= 256 else (1,)), s
            else:
                assert s["multipass"] == 0
            if ragged:
                assert C <= 8
            if C > 8:
                assert 16 <= C <= 512
                if s["multipass"] == 2:
                    assert (4096 // C) * (8 if prec == FP32 else 16) % 16 == 0  # box rows
                continue
            LC, es = 1 << lc, (8 if prec == FP32 else 16)
            S0 = LC // R
            assert S0 % NT == 0 and S0 // NT >= 1, s  # pass-0 groups divide over threads
            assert len(_passes(lc, R)) >= 2
            if C > 1:
                assert (LC // C) % (2 * NT) == 0, s  # cross stage: two positions per thread
            assert NT * s["MINB"] <= 2048 and 65536 // (NT * s["MINB"]) >= 32
            assert LC * es + (LC // 2) * es <= SMEM_MAX  # FFT buffer and scaled input
    assert seen_any > 20


def test_radix32_variants_are_candidates(tdh):
    """2^14 ... 2^17 float32 points (1, 2, 4, 8 slices of 2^14) default to the radix-32
    kernel, with the radix-16 one as a candidate, dense and ragged; float64 has none;
    single-CTA 2^13-point FFTs have a radix-32 candidate."""
    for logL in (14, 15, 16, 17):
        for ragged in (False, True):
            sched = tdh.compiled_schedules(FP32, logL, ragged)
            assert (sched[0]["logLC"], sched[0]["R"]) == (14, 32), (logL, sched[0])
            rs = [s["R"] for s in sched if s["logLC"] == 14 and s["NT"] == 512]
            assert sorted(rs) == [16, 32], (logL, ragged, rs)
        assert all(s["R"] != 32 for s in tdh.compiled_schedules(FP64, logL))
    # single-CTA FFTs of 2^13 and 2^14 points have radix-32 candidates too
    for logL, nt in ((13, 256), (14, 512)):
        assert any(s["R"] == 32 and s["C"] == 1 and s["NT"] == nt
                   for s in tdh.compiled_schedules(FP32, logL)), logL


def test_lengths_without_a_kernel(tdh):
    """Beyond 512 slices nothing is compiled; ragged batches stop at one cluster."""
    assert tdh.compiled_schedules(FP32, 24) == []
    assert tdh.compiled_schedules(FP64, 23) == []
    assert tdh.compiled_schedules(FP32, 18, ragged=True) == []
    assert tdh.compiled_schedules(FP32, 17, ragged=True)[0]["C"] == 8


def test_bad_arguments(tdh):
    import ctypes
    n = ctypes.c_int()
    assert tdh.lib().tdh_schedules(7, 10, 0, None, 0, ctypes.byref(n)) == -1
    assert tdh.lib().tdh_schedules(FP32, 0, 0, None, 0, ctypes.byref(n)) == -1
    assert tdh.lib().tdh_schedules(FP32, 10, 0, None, 3, ctypes.byref(n)) == -1
