"""Host-side logic without a GPU: multi-rank aggregation of the benchmark
(world size 2 over gloo) and the seeded request streams of the served loop."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total, fwd, rays = bench.reduce_over_ranks(100.0 + 50 * rank, 10.0 * (rank + 1), 1000 * (rank + 1), "cpu")
    out[rank] = (total, fwd, rays)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_and_rays_are_summed_over_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (150.0, 20.0, 3000.0)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 3.0, 77, "cpu") == (12.5, 3.0, 77.0)


def test_request_stream_is_seeded_poisson_with_valid_edits():
    from synthetic import scenes as S
    from synthetic.requests import request_stream
    sc = S.scene_c2(0, per_face=200, per_object=300)
    a = request_stream(400, 5.0, sc, seed=1)
    b = request_stream(400, 5.0, sc, seed=1)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 0.2) < 0.03 and np.all(gaps > 0)
    kinds = {r.edit["kind"] for r in a}
    assert kinds == {"move", "material", "env"}
    for r in a:
        if r.edit["kind"] == "move":
            R = r.edit["R"].astype(np.float64)
            assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and abs(np.linalg.det(R) - 1) < 1e-6
            assert 1 <= r.edit["object"] < sc.n_objects
        assert r.cam.width in (256, 512, 800, 1024) and r.spp in (4, 8, 16, 32)


def test_inverse_rendering_schedule():
    from paper_2608_29269_b300.render import spp_schedule as sched, trainable_groups as groups
    assert [sched(i) for i in (0, 7499, 7500, 11999, 12000, 14999)] == [8, 8, 16, 16, 32, 32]
    assert groups(0) == ("env",) and groups(1999) == ("env",)
    assert groups(2000) == ("env", "albedo") and groups(8999) == ("env", "albedo")
    assert groups(9000) == ("env", "albedo", "metallic", "roughness")


def test_checkpoint_round_trip_on_the_host(tmp_path):
    """Scene, environments, constants, per-state transforms and the replay
    seed survive a save / load unchanged (CPU tensors, no library call)."""
    import torch
    from paper_2608_29269_b300 import SceneTensors, load_checkpoint, save_checkpoint
    from paper_2608_29269_b300._native import LfParams
    from synthetic import scenes as S
    sc = S.scene_c2(0, per_face=200, per_object=300)
    st = SceneTensors.from_numpy(sc, device="cpu")
    envs = {0: torch.as_tensor(S.env_sky_sun(0, H=16, W=32).rgb), 3: torch.full((8, 16, 3), 0.5)}
    p = LfParams()
    p.T_min, p.alpha_min, p.max_rounds, p.sampler = 1e-4, 1.0 / 255.0, 64, 1
    rng = np.random.default_rng(0)
    R = np.stack([S.rigid_motion(rng, np.zeros(3))[0] for _ in range(sc.n_objects - 1)])
    t = rng.normal(size=(sc.n_objects - 1, 3)).astype(np.float32)
    path = tmp_path / "scene.npz"
    save_checkpoint(path, st, envs=envs, params=p, states={"layout 3": (R, t)}, seed=1234, spp=16)
    ck = load_checkpoint(path, device="cpu")
    for k in ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic", "roughness"]:
        assert torch.equal(getattr(ck.scene, k), getattr(st, k)), k
    assert list(ck.scene.object_offsets) == [int(v) for v in sc.object_offsets]
    assert sorted(ck.envs) == [0, 3] and all(torch.equal(ck.envs[s], envs[s]) for s in envs)
    assert ck.params["max_rounds"] == 64 and ck.params["sampler"] == 1
    assert ck.params["T_min"] == np.float32(1e-4) and ck.lf_params().alpha_min == np.float32(1.0 / 255.0)
    np.testing.assert_array_equal(ck.states["layout 3"][0], R)
    np.testing.assert_array_equal(ck.states["layout 3"][1], t)
    assert ck.seed == 1234 and ck.spp == 16
    # a file whose offsets do not partition the surfels is refused
    bad = SceneTensors(**{k: getattr(st, k) for k in ["mu", "tu", "tv", "scale", "opacity", "albedo", "metallic",
                                                     "roughness"]}, object_offsets=[0, 5, 3, sc.n])
    save_checkpoint(tmp_path / "bad.npz", bad)
    with pytest.raises(ValueError):
        load_checkpoint(tmp_path / "bad.npz", device="cpu")
