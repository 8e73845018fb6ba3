"""Physics performance of the GPU's tracks equals that of the oracle's on
the same events (the selections are identical), and is reported."""
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_gpu_and_oracle_tracks_give_the_same_physics_performance():
    import paper_2002_11529_gb300 as g
    from paper_2002_11529_gb300 import physics
    g.build.build()
    b = synth.generate_config("plain", n_events=50)
    P = synth.CompassParams()
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, P)
    pipe.run_batched()
    ctx.check(what="physics")
    gpu = physics.evaluate(b, g.tracks_to_numpy(pipe.tracks, b.n_tracks))
    _, orc = oracle.run_batch(b, P)
    ref = physics.evaluate(b, {"hit": orc.hit, "found": orc.found})
    print(f"\nefficiency {gpu['efficiency']:.4f}, fake rate {gpu['fake_rate']:.4f} "
          f"({gpu['reconstructible']} reconstructible, {gpu['found']} found)")
    assert gpu == ref
