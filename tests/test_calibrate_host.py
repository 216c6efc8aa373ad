"""The model recalibration's fit, without a GPU: on times generated by the
model itself from known terms, the fit reaches them (near-zero residual) and
its picks are those of the generating terms."""
import json

import pytest

from paper_2301_03598_gb300 import build, calibrate, inputs
from paper_2301_03598_gb300 import streamk as sk

pytest.importorskip("scipy")


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def synthetic(path, coefs, count=60, num_sms=152):
    shapes = inputs.sweep_shapes(count)
    data = {"num_sms": num_sms, "shapes": shapes, "plans": {}}
    for tn, cm in calibrate.CONFIGS:
        for mode in calibrate.MODES:
            us, plans = [], []
            for (m, n, k) in shapes:
                info = sk.sk_plan_describe(m, n, k, mode, tile_n=tn, cluster_m=cm, num_sms=num_sms)
                plans.append([info["mode"], info["grid"], info["sk_tiles"], info["dp_tiles"],
                              info["workspace_bytes"]])
                us.append(sk.sk_model_time(m, n, k, mode, tile_n=tn, cluster_m=cm, num_sms=num_sms,
                                           grid=info["grid"] if mode == "sk" else 0,
                                           coef=coefs[f"{tn}x{cm}"]))
            data["plans"][f"{mode}/{tn}x{cm}"] = {"us": us, "plan": plans}
    with open(path, "w") as f:
        json.dump(data, f)
    return data


def test_fit_recovers_model_generated_times(tmp_path, capsys):
    true = {f"{tn}x{cm}": [v * s for v, s in zip(sk.sk_model_coefficients(tn, cm),
                                                 (1.2, 0.7, 1.1, 1.3, 0.8, 0.9))]
            for tn, cm in calibrate.CONFIGS}
    data = synthetic(tmp_path / "cal.json", true)
    calibrate.main(["fit", str(tmp_path / "cal.json"), "--out", str(tmp_path / "fit.json")])
    out = capsys.readouterr().out
    for line in out.splitlines():
        if "rms log error" in line:
            assert float(line.split("->")[1]) < 2e-3, line
    fitted = json.load(open(tmp_path / "fit.json"))
    # the fitted terms make the generating terms' picks (which differ from the
    # best measured plan only where the 10% split margin declines a split)
    q, _ = calibrate.pick_quality(sk, data, true, ["dp", "hybrid", "sk"])
    assert 1.0 <= q < 1.01
    assert fitted["pick_quality"]["fitted"] == pytest.approx(q, abs=1e-3)
