"""GB300-native RadioPropa ray-propagation hot path (package placeholder; binding follows)."""
