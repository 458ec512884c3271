"""Host-side helpers of bench.py on CPU: the clock record of the timed region
and the samplers' behaviour where no GPU tool is present."""
import bench


def test_clock_record_prefers_nvml_samples_and_unions_reasons():
    smi = {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 1}
    nv = {"nvml_sm_mhz": 2070.0, "nvml_sm_max_mhz": 2070, "nvml_reasons": ["hw_slowdown"],
          "nvml_samples": 40}
    c = bench.merge_clocks(smi, nv)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert c["samples"] == 41 and c["smi_samples"] == 1 and c["nvml_samples"] == 40


def test_clock_record_without_nvml_keeps_nvidia_smi():
    smi = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    c = bench.merge_clocks(smi, {"nvml_samples": 0})
    assert c["sm_mhz"] == 2070.0 and c["samples"] == 3 and c["reasons"] == []


def test_nvml_reason_bits():
    s = bench.NvmlSampler.__new__(bench.NvmlSampler)
    s.samples = [(2070, 2070, 0x4), (2070, 2070, 0), (1500, 2070, 0x8 | 0x40)]
    out = s.summary()
    assert out["nvml_reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert out["nvml_sm_mhz"] == 2070 and out["nvml_samples"] == 3


def test_samplers_without_gpu_tools_record_nothing():
    with bench.ClockSampler(0) as smi, bench.NvmlSampler(0) as nv:
        pass
    assert isinstance(smi.summary(), dict)
    assert nv.summary().get("nvml_samples", 0) >= 0
